// Persistent step of a p-adaptive batch: one cooperative launch per step.  Every CTA
// claims work items (element group, tile) from an atomic counter, first the local phase
// of all groups (derivatives, time integral, volume, face projections, local flux
// products), then, after a grid-wide barrier, the neighbour phase (neighbour flux and
// lifting).  The per-degree work of a tile is the same code as the kernels of a single
// solver (local_tile / neigh_tile), compiled per degree and contraction type in
// separately compiled translation units and called through a switch on the degree.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "ader_kernels.cuh"

namespace yt {

// One element group of the batch (all elements of one degree), as its tiles are computed.
struct BatchGroup {
  int N;                     // polynomial degree
  double *Q, *I;             // [tile][9][B][32]
  void *Pface, *Wloc;        // contraction type
  const void *star, *floc, *fnb;
  const int* conn;           // packed cross-group connectivity
  const void *val, *f;       // global-matrix values and f^h of this degree
  double dt;
};

struct BatchArgs {
  const BatchGroup* groups;  // device array
  FaceGroups faces;          // face projections of every group (neighbour gathers)
  const int2* items;         // [n_items[0] local items][n_items[1] neighbour items]: (group, tile)
  int n_items[2];
  int chunk;                 // items per claim
  int* counters;             // [0] local claims, [1] neighbour claims, [2] barrier arrivals
  int* status;               // YT_ERR_TIMEOUT when the barrier wait ran out
  StarPattern SP;
};

constexpr unsigned long long kBarrierWaitNs = 1000000000ull;   // 1 s

// Host side (batch_rdc.cu): dynamic shared memory attribute, occupancy (CTAs per SM) and
// launch (cooperative when `cooperative`) of the persistent kernel of one contraction type.
int batch_persistent_prepare(bool f32, size_t smem);
cudaError_t batch_persistent_launch(bool f32, const BatchArgs& A, unsigned grid, size_t smem,
                                    cudaStream_t st, bool cooperative);

}  // namespace yt
