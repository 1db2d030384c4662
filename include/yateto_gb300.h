/*
 * yateto_gb300 — C ABI of a GB300 (sm_103a) library for the element kernels of
 * tetrahedral ADER-DG (Uphoff & Bader, "Yet Another Tensor Toolbox for discontinuous
 * Galerkin methods and other applications", arXiv 1903.11521).
 *
 * Two layers:
 *   1. Planner + batched executor for small tensor contractions written in Einstein
 *      notation (Sec. 4): yt_plan_create / yt_plan_stats_get / yt_plan_eqspp /
 *      yt_execute_batched / yt_plan_destroy.
 *   2. A fused solver for one elastic ADER-DG step (Sec. 5.1, Eqs. seissol:derivative,
 *      seissol:timeint, seissol:correction_local, seissol:correction_neigh):
 *      yt_solver_create / yt_solver_set_dofs / yt_solver_get / yt_step /
 *      yt_step_local / yt_step_neighbour / yt_solver_destroy.
 *
 * Conventions for every entry point:
 *   - Every call returns a yt_status; no exception or abort crosses the ABI.  After an
 *     error, yt_last_error() returns a message for the calling thread.
 *   - Device work is enqueued asynchronously on the given stream (0 = legacy default
 *     stream); nothing synchronises unless stated.  A pointer marked "host" must be host
 *     memory, "device" must be device memory of the current device.
 *   - Tensors are column-major (first index fastest, Sec. 4.4, dense layout).
 *   - Plans and solvers are owned by the library and freed by their destroy call.
 *     Caller-provided buffers stay owned by the caller.
 *   - A plan is immutable after creation and may be used from several threads; a solver
 *     must not be stepped concurrently from several threads.
 * There is no CPU fallback: without a CUDA device, calls that launch kernels return
 * YT_ERR_CUDA.
 */
#ifndef YATETO_GB300_H
#define YATETO_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* yt_stream;   /* same type as cudaStream_t */

typedef enum yt_status {
  YT_OK = 0,
  YT_ERR_INVALID = 1,      /* null pointer, out-of-range argument */
  YT_ERR_PARSE = 2,        /* malformed Einstein expression */
  YT_ERR_SHAPE = 3,        /* inconsistent index sizes / tensor dimensions */
  YT_ERR_UNSUPPORTED = 4,  /* valid request that the library has no kernel for */
  YT_ERR_OOM = 5,          /* device or host allocation failed */
  YT_ERR_CUDA = 6,         /* a CUDA runtime call failed (incl. no device) */
  YT_ERR_TIMEOUT = 7       /* a bounded device-side wait ran out */
} yt_status;

typedef enum yt_precision {
  YT_F64 = 0,              /* all arithmetic in binary64 */
  YT_F32 = 1,              /* bulk contractions in binary32, setup in binary64 */
  YT_BF16X3_F32ACC = 2     /* products with the global matrices on the tensor cores: each
                              operand split into two bfloat16 parts (hi + lo), three
                              products hi*hi + hi*lo + lo*hi accumulated in binary32;
                              per-element 9x9 products in binary32, DOFs and time-integral
                              accumulation in binary64 (solver only, orders 2..7) */
} yt_precision;

typedef enum yt_memory { YT_MEM_HOST = 0, YT_MEM_DEVICE = 1 } yt_memory;

typedef enum yt_field {
  YT_FIELD_DOFS = 0,             /* Q, the degrees of freedom */
  YT_FIELD_TIME_INTEGRAL = 1     /* I, the time-integrated DOFs of the last step */
} yt_field;

/* ------------------------------------------------------------------ diagnostics */
const char* yt_status_string(yt_status s);
/* Message of the last failing call on this thread ("" if none).  Valid until the next
 * failing call on the same thread. */
const char* yt_last_error(void);
/* Library version string, e.g. "yateto_gb300 0.1 sm_103a". */
const char* yt_version(void);

/* ===================================================================== planner
 *
 * yt_plan_create parses an assignment in the DSL of Sec. 4.1
 *     "Q[kp] += Kh[kl] * I[lq] * As[pq]"
 *     "C[ij] = 2.0 * A[lj] * B[ikl] * w[k]"
 *     "Q[kp] += Kx[kl] * I[lq] * Ax[pq] + Ky[kl] * I[lq] * Ay[pq]"
 * LHS "=" or "+="; the RHS is a sum of terms, each an optional numeric scalar followed by
 * a product of indexed tensors.  Index letters [a-zA-Z]; each tensor's index string must
 * have one letter per dimension and no repeated letter (Sec. 4.2.1: the trace T_ii is not
 * an Einstein product here).  Every letter of a term that is not on the LHS is summed.
 * For every term the planner computes the equivalent sparsity patterns (Eq. compeqspp),
 * the operation-minimal binary tree under the sparse cost of Sec. 4.3, the index
 * permutations of the temporaries by the dynamic program of Sec. 4.5 (Eqs. permopt,
 * permcost, subproblem) with the Loop-over-GEMM cost (s, l+r, -f), and the non-zero flop
 * count.  A stored value 0.0 of a global constant is treated as a structural zero.
 * yt_plan_create, yt_plan_stats_get and yt_plan_eqspp run on the host only; the plan's
 * device tables are created by its first yt_execute_batched.
 */
typedef struct yt_tensor_desc {
  const char* name;         /* as used in the expression */
  int32_t ndim;             /* 0..8 */
  const int32_t* shape;     /* host, ndim entries */
  const uint8_t* pattern;   /* host, column-major boolean non-zero pattern of prod(shape)
                               bytes; NULL = dense */
  const double* values;     /* host, column-major values of a global constant (uploaded
                               and owned by the plan); NULL = per-element tensor */
} yt_tensor_desc;

typedef struct yt_plan_stats {
  double nz_flops;           /* non-zero flops per element (Sec. 4.9) */
  double hw_flops;           /* flops the executor performs per element */
  double naive_flops;        /* cost of the unreduced n-ary product per element */
  int64_t bytes_per_element; /* per-element tensor bytes read + written */
  int32_t n_ops;             /* binary operations after strength reduction */
  int32_t n_terms;
  int64_t log_cost[4];       /* Loop-over-GEMM cost (s, l+r, -f, l) of the chosen index
                                orders, summed over all binary nodes of all terms */
  char order[1024];          /* the trees, e.g. "sum_l(A[lj]*sum_k(B[ikl]*w[k])[il])[ij]":
                                "sum_x(L*R)[o]" multiplies L and R, sums the indices x and
                                stores the result in index order o */
} yt_plan_stats;

struct yt_plan;

yt_status yt_plan_create(const char* expr, const yt_tensor_desc* tensors,
                         int32_t n_tensors, yt_precision precision,
                         struct yt_plan** out_plan);
yt_status yt_plan_stats_get(const struct yt_plan* plan, yt_plan_stats* out);
/* Equivalent sparsity pattern (Eq. compeqspp) of tensor `tensor_index` (position in the
 * descriptor array) within term `term`; writes prod(shape) bytes (host, column-major). */
yt_status yt_plan_eqspp(const struct yt_plan* plan, int32_t term, int32_t tensor_index,
                        uint8_t* pattern_out);
/* Runs the plan for n_elements elements.  element_tensors[i] is the device pointer of
 * descriptor i if that descriptor is per-element (values == NULL), ignored otherwise.
 * Per-element tensors are stored element after element, each dense column-major in the
 * plan's precision (double for YT_F64, float for YT_F32).  The LHS tensor is read only
 * for "+=".  Scratch for temporaries is allocated by the plan on first use. */
yt_status yt_execute_batched(const struct yt_plan* plan, void* const* element_tensors,
                             int64_t n_elements, yt_stream stream);
/* Allocation-free variant of yt_execute_batched (the paper has no counterpart).
 * For callers that must not allocate device memory themselves or through libraries they
 * call: code whose device memory is owned by a host framework's own pool, or loops that
 * must not take the device-wide synchronisation that cudaMalloc / cudaFree can imply.
 * Same arguments and results as yt_execute_batched (up to the summation order): it always
 * runs the lane-per-element executor kernel with the temporaries in global scratch, also
 * for plans that yt_execute_batched runs on its element-per-warp kernel with the
 * temporaries in shared memory, so its speed can differ.  It calls no cudaMalloc, cudaFree or
 * allocating routine: the plan's operation list, index lists, constants and the
 * temporaries live in fixed arrays inside the library (reserved on every device that
 * loads it, until process exit): temporaries 32 MiB, index lists 2^20 integers, 4096
 * operations, constants 2 MiB.  A plan beyond any of these limits is rejected with
 * YT_ERR_UNSUPPORTED and a message naming the limit; nothing runs then.  The first call
 * on each device looks up the arrays' device addresses (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.  Every call copies the
 * plan's tables into the shared arrays (from host copies that the plan owns, on `stream`)
 * and then runs the kernel; calls whose work overlaps on the device, e.g. on two streams, race on the
 * shared arrays and must be serialised by the caller. */
yt_status yt_execute_batched_noalloc(const struct yt_plan* plan, void* const* element_tensors,
                                     int64_t n_elements, yt_stream stream);
void yt_plan_destroy(struct yt_plan* plan);

/* ===================================================================== solver
 *
 * Elastic ADER-DG on tetrahedra (Sec. 5.1).  Quantities q = (sxx, syy, szz, sxy, syz,
 * sxz, u, v, w); polynomial degree N = order - 1; B = C(N+3,3) Dubiner basis functions
 * (degree-major, then lexicographic in (p, q) of phi_pqr).
 *
 * Per step (all on the device):
 *   D^0 = Q,  D^{d+1} = sum_x Ktilde^x D^d Astar^x^T                (CK derivatives)
 *   I = sum_{d=0}^{N} dt^{d+1}/(d+1)! D^d                          (time integral)
 *   Q += sum_x Khat^x I Astar^x^T + sum_s Rhat^s R^sT I Aloc_s^T     (volume + local flux)
 *   Q += sum_s Rhat^s f^h R^jT I_nb Anb_s^T,  (nb, j, h) = neighbour, its face, orientation
 * with Khat^x = M^-1 K^x, Ktilde^x = -M^-1 K^xT, K^x_kl = int dphi_k/dxi_x phi_l,
 * Astar^x = sum_j (dxi_x/dx_j) A^j and upwind flux solvers
 * Aloc_s = -(2|S_s|/|J|)(A_n + |A_n|)/2, Anb_s = -(2|S_s|/|J|)(A_n - |A_n|)/2.
 */
typedef struct yt_mesh_desc {
  int64_t n_elements;
  const double* material;    /* host, E x 3: rho, lambda, mu per element */
  const double* jacobian;    /* host, E x 9: dx/dxi of the affine map, column-major 3x3
                                (column c = physical edge vector x_c - x_0) */
  const int32_t* neighbours; /* host, E x 4: element behind face s (0..E-1), or NULL for
                                a local-only solver (yt_step_neighbour then fails) */
  const int8_t* faces;       /* host, E x 4: the neighbour's face index j (0..3) */
  const int8_t* orient;      /* host, E x 4: orientation h (0..2) */
  const double* attenuation; /* host, E x 3 x 3: (omega_l, Y^lambda_l, Y^mu_l) of the
                                mechanisms l = 0..2, for 27-quantity solvers; else NULL */
  int64_t n_halo;            /* partitioned solves: number of halo slots (else 0); a
                                neighbour entry -1 - t (t < n_halo) means that face's
                                neighbour lives on another rank and its face projection
                                is slot t of the halo block (yt_solver_halo_buffer) */
} yt_mesh_desc;

typedef struct yt_scheme_desc {
  int32_t order;             /* convergence order O = N + 1: 2..7 */
  double dt;                 /* time step */
  yt_precision precision;    /* YT_F64, YT_F32 or YT_BF16X3_F32ACC (orders 2..7) */
  int32_t flags;             /* 0, or YT_SCHEME_DIAG_EXPIRE_WAIT */
  int32_t quantities;        /* 9 (or 0): elastic; 27: viscoelastic-shaped (below) */
} yt_scheme_desc;
/* 27-quantity solvers (YT_F64, YT_F32 or YT_BF16X3_F32ACC, orders 2..7).  The paper names viscoelastic
 * attenuation with three mechanisms (27 quantities, Sec. 5.1) without its equations; this
 * library reads it as the memory-variable form q = (sigma, v, theta^0, theta^1, theta^2),
 * q_t + A q_x + B q_y + C q_z = E q, with six anelastic functions theta^l per mechanism:
 *   - the rows of theta^l in A, B, C are omega_l times the stress-velocity rows of the
 *     elastic Jacobian with the moduli (Y^lambda_l, Y^mu_l); their columns are zero;
 *   - E: d sigma_i/dt gets -sum_l theta^l_i, d theta^l_i/dt gets -omega_l theta^l_i.
 * The step is the elastic one with D^{d+1} += D^d E^T in the CK recursion and Q += I E^T
 * in the update (the source enters through the time-integrated DOFs); star matrices and
 * upwind flux solvers are those of the 27 x 27 Jacobians (|A_n| = a A_n^2 + b A_n^4 on
 * the same spectrum).  Quantity order in every DOF array: the 9 elastic ones, then
 * theta^l_i at 9 + 6 l + i.  yt_step, yt_step_phase (phase 1 runs two kernels: the
 * elastic neighbour flux and the anelastic rows' volume, source and fluxes) and
 * yt_step_host are available; yt_step_local / yt_step_neighbour, batches and servers are
 * elastic only (YT_ERR_UNSUPPORTED).  With YT_BF16X3_F32ACC the elastic rows' products
 * with the global matrices run on the tensor cores (split bf16), the anelastic functions'
 * derivatives on the CUDA cores in FP32 inside the same local kernel, and the anelastic
 * rows' volume, source and fluxes in the FP32 kernel of YT_F32; setup, the time integral
 * and the DOF updates in binary64 as for every precision. */
/* Diagnostics flag (no counterpart in the paper), YT_BF16X3_F32ACC solvers only: the
 * tensor-core local kernel does not issue its operand load and its first bounded wait
 * (on that load) gives up after 1 ms, before any tensor-core or bulk-copy operation is
 * in flight; the kernel then issues nothing, frees its tensor memory and records the
 * timeout, which yt_solver_status reports as YT_ERR_TIMEOUT.  The outputs of such a step
 * are meaningless.  For testing the timeout path without a fault or a hang. */
#define YT_SCHEME_DIAG_EXPIRE_WAIT 1

struct yt_solver;

/* Builds the reference matrices, uploads material, geometry and connectivity and runs
 * the per-element setup kernel (star matrices, flux solvers) on `stream`.  Device memory
 * is allocated here; DOFs start at zero. */
yt_status yt_solver_create(const yt_mesh_desc* mesh, const yt_scheme_desc* scheme,
                           yt_stream stream, struct yt_solver** out_solver);
/* Copies Q in: `dofs` holds E x P x B values (P = the solver's quantities, 9 or 27) in
 * the canonical element layout [element][quantity][basis] (basis index fastest,
 * column-major B x P per element), as double, in host or device memory (`where`).  Asynchronous on `stream`; host memory must
 * stay valid until the stream reaches this point (use pinned memory to overlap). */
yt_status yt_solver_set_dofs(struct yt_solver* solver, const double* dofs, yt_memory where,
                             yt_stream stream);
/* Copies a field out in the canonical layout (as above), as double. */
yt_status yt_solver_get(struct yt_solver* solver, yt_field field, double* out,
                        yt_memory where, yt_stream stream);
/* One full step: the local kernel (derivatives, time integral, volume, local flux),
 * then the neighbour kernel. */
yt_status yt_step(struct yt_solver* solver, yt_stream stream);
/* Partial updates: yt_step_local applies derivatives, time integral, volume and local
 * flux (the complete local update); yt_step_neighbour then applies the neighbour flux.
 * Together they give the same result as yt_step up to rounding.  A YT_F64 / YT_F32
 * solver of orders 2..5 whose mesh has at most one tile of 32 elements per SM runs
 * yt_step_local on CTAs of 8 elements (the same arithmetic, bitwise the same result). */
yt_status yt_step_local(struct yt_solver* solver, yt_stream stream);
yt_status yt_step_neighbour(struct yt_solver* solver, yt_stream stream);
/* The two kernels of yt_step, one at a time (phase 0 then phase 1 == yt_step): phase 0
 * computes derivatives, time integral, volume, the face projections and the local flux
 * products (R^sT I) Aloc_s^T; phase 1 adds the neighbour products and applies
 * Rhat^s once per face to their sum.  Q is only consistent after phase 1. */
yt_status yt_step_phase(struct yt_solver* solver, int32_t phase, yt_stream stream);
/* One step (as yt_step) on host buffers: Q is read from `dofs_in` and the new Q written to
 * `dofs_out` (host memory, canonical layout; they may be the same buffer).  The transfers
 * are pipelined with the kernels in up to 16 element chunks (each a whole number of
 * waves of one CTA per SM where the mesh allows) on an internal copy stream: the
 * upload of a chunk overlaps the local kernel of the previous one, and the download of a
 * chunk overlaps the neighbour kernel of the next one (the neighbour kernel of any chunk
 * needs the local results of all chunks).  Host buffers should be pinned for the copies
 * to run asynchronously.  Asynchronous on `stream`: the step, including the last
 * download, is complete when `stream` reaches this point.  The time integral stays on
 * the device (yt_solver_get). */
yt_status yt_step_host(struct yt_solver* solver, const double* dofs_in, double* dofs_out,
                       yt_stream stream);
/* ---------------------------------------------------------------- partitioned solves
 * The step shards by elements with one exchange per step: after phase 0 every rank holds
 * the face projections R^jT I of its own elements; phase 1 of an element whose face
 * neighbour lives on another rank reads that neighbour's projection from the halo block
 * (mesh->n_halo slots, BT x 9 values each in the contraction type, laid out
 * [slot][quantity][BT]).  Per step: yt_step_phase(0); yt_solver_halo_pack (gathers the
 * projections that other ranks need, in the order of the send list); the transfer
 * (NCCL, peer copies or host staging: the caller's) into yt_solver_halo_buffer;
 * yt_step_phase_tiles(1) on the tiles without remote neighbours may run while it is in
 * flight; then phase 1 on the other tiles.  Elastic YT_F64 / YT_F32 solvers only. */
/* Sets the send list: n_pairs (local element, face j) pairs (host, int32 x 2 each). */
yt_status yt_solver_set_send_list(struct yt_solver* solver, const int32_t* pairs, int64_t n_pairs);
/* Gathers the projections of the send list (after phase 0) into `out` (device,
 * n_pairs x 9 x BT values of the contraction type), on `stream`. */
yt_status yt_solver_halo_pack(struct yt_solver* solver, void* out, yt_stream stream);
/* Device address and size in bytes of the halo block (receive into it before phase 1). */
yt_status yt_solver_halo_buffer(struct yt_solver* solver, void** ptr, int64_t* bytes);
/* Copies n_halo x 9 x BT values (device memory, contraction type) into the halo block on
 * `stream` (for receive buffers that the caller owns). */
yt_status yt_solver_halo_unpack(struct yt_solver* solver, const void* in, yt_stream stream);
/* One phase (0 or 1, as yt_step_phase) of the fused step over tiles [tile0, tile0 + n)
 * (tiles of 32 consecutive elements); phase 1 of a tile needs phase 0 of every tile and
 * the halo.  The number of tiles is ceil(E / 32). */
yt_status yt_step_phase_tiles(struct yt_solver* solver, int32_t phase, int64_t tile0, int64_t n_tiles,
                              yt_stream stream);

/* Flops per element executed by the two phases of yt_step, and their algorithmic device
 * bytes per element (each stream read or written once). */
yt_status yt_solver_stats(const struct yt_solver* solver, double* local_flops,
                          double* neighbour_flops, double* local_bytes,
                          double* neighbour_bytes);
/* Synchronises `stream`, then reports whether a bounded device-side wait of this solver's
 * kernels ran out since the last call: the tensor-core kernels (YT_BF16X3_F32ACC) wait on
 * tensor-core completion with a limit of one second and then stop with their outputs
 * incomplete.  Returns YT_ERR_TIMEOUT (and clears the record) in that case, else YT_OK.
 * No counterpart in the paper: a safeguard of this implementation. */
yt_status yt_solver_status(struct yt_solver* solver, yt_stream stream);
/* Reference matrix `name` ("M", "Khat", "Ktilde", "R", "Rhat", "f") of this solver's
 * order as double, column-major, stacked over its first index (3, 4 or 3 matrices);
 * `count` receives the number of doubles; pass out == NULL to query the size. */
yt_status yt_solver_reference_matrix(const struct yt_solver* solver, const char* name,
                                     double* out, int64_t* count);
void yt_solver_destroy(struct yt_solver* solver);

/* ------------------------------------------------------------- p-adaptive batches
 * Elements of different polynomial degrees in one mesh (orders 2..7 per element, YT_F64
 * or YT_F32).  Each element uses its own degree for derivatives, time integral,
 * volume and local flux; across a face, the neighbour's face projection is truncated or
 * zero-padded to the element's face basis (the hierarchical orthogonal basis makes this
 * the L2 projection).  The elements are grouped by degree; one step is one launch of a
 * CUDA graph recorded at creation (see the forms below).  DOFs are exchanged in the packed canonical layout: element after
 * element (in mesh order), each [quantity][basis] with its own B_e = C(o_e + 2, 3). */
struct yt_batch;
yt_status yt_batch_create(const yt_mesh_desc* mesh, const int8_t* orders /* host, E */,
                          const yt_scheme_desc* scheme /* order ignored */, yt_stream stream,
                          struct yt_batch** out_batch);
yt_status yt_batch_set_dofs(struct yt_batch* batch, const double* dofs, yt_memory where,
                            yt_stream stream);
yt_status yt_batch_get(struct yt_batch* batch, yt_field field, double* out, yt_memory where,
                       yt_stream stream);
yt_status yt_batch_step(struct yt_batch* batch, yt_stream stream);
/* Forms of the step (each recorded as one CUDA graph, one graph launch per step):
 *   0: the per-degree local kernels in sequence, then the neighbour kernels;
 *   1: the same kernels on parallel graph branches (one branch per degree);
 *   2: one persistent kernel: a cooperative launch of one CTA per SM (as many as the
 *      occupancy query allows) in which every CTA claims work items (degree group, tile)
 *      from an atomic counter, `chunk` tiles per claim, in one of two orders (0: groups by
 *      decreasing degree, the longest tiles first; 1: groups interleaved tile by tile);
 *      the local phase of every group, then a grid-wide barrier (bounded wait, one
 *      second, then YT_ERR_TIMEOUT through yt_batch_status), then the neighbour phase.
 * A new batch uses form 0.  yt_batch_set_form selects a form (order and chunk apply to
 * form 2). */
yt_status yt_batch_set_form(struct yt_batch* batch, int32_t form, int32_t order, int32_t chunk);
/* Autotuner: records every form (0, 1, and 2 with each order and chunk 1, 2, 4), replays
 * each `repeats` times on the current data (the DOFs are restored afterwards), keeps the
 * fastest and reports its form in *chosen.  Synchronises `stream`. */
yt_status yt_batch_tune(struct yt_batch* batch, int32_t repeats, yt_stream stream, int32_t* chosen);
/* Description of the form in use (and the tuner's timings after yt_batch_tune), as a
 * NUL-terminated string of at most capacity - 1 characters. */
yt_status yt_batch_config(const struct yt_batch* batch, char* out, int32_t capacity);
/* Synchronises `stream`, then reports whether the persistent kernel's grid barrier ran
 * out since the last call (YT_ERR_TIMEOUT, record cleared), else YT_OK.  No counterpart
 * in the paper: a safeguard of this implementation. */
yt_status yt_batch_status(struct yt_batch* batch, yt_stream stream);
/* Flops and algorithmic device bytes of one step of the whole batch; number of groups. */
yt_status yt_batch_stats(const struct yt_batch* batch, double* flops, double* bytes,
                         int32_t* n_groups);
void yt_batch_destroy(struct yt_batch* batch);

/* ------------------------------------------------------------------ serving
 * Independent solves (own mesh, order, dt, DOFs and number of steps) submitted at any
 * time.  A worker thread admits pending requests in arrival order while the device memory
 * of the admitted solves fits `hbm_budget_bytes` (a request larger than the whole budget
 * fails with YT_ERR_OOM), and advances all admitted solves together: each step of the
 * server runs, per polynomial degree, one local and one neighbour kernel over the tiles
 * of all admitted solves of that degree, the degrees on separate streams.  A finished
 * solve is copied out and freed at once, and requests that arrived meanwhile are admitted
 * as memory frees up.  Results are identical to those of the same solve alone.  The
 * server uses the device that is current at yt_server_create. */
typedef struct yt_server_desc {
  int64_t hbm_budget_bytes;
  yt_precision precision;    /* YT_F64 or YT_F32 (orders 2..7) */
  int32_t flags;             /* reserved, must be 0 */
} yt_server_desc;

typedef struct yt_server_stats {
  int64_t submitted, completed, failed, pending, active, max_active, ticks;
  int64_t budget_bytes, peak_bytes;  /* peak = most device memory admitted at once */
  double element_updates;            /* element-steps completed so far */
} yt_server_stats;

struct yt_server;
yt_status yt_server_create(const yt_server_desc* desc, struct yt_server** out_server);
/* Copies the inputs (host memory; DOFs in the canonical layout) and queues the request;
 * returns at once with its id. */
yt_status yt_server_submit(struct yt_server* server, const yt_mesh_desc* mesh, int32_t order,
                           double dt, const double* dofs, int32_t n_steps,
                           int64_t* request_id);
/* Blocks until the request is done; copies its final DOFs (canonical layout, host) to
 * dofs_out unless NULL; latency_s = completion - submission, queue_s = admission -
 * submission.  Returns the request's error if it failed. */
yt_status yt_server_wait(struct yt_server* server, int64_t request_id, double* dofs_out,
                         double* latency_s, double* queue_s);
yt_status yt_server_stats_get(struct yt_server* server, yt_server_stats* out);
/* Finishes every submitted request, then stops the worker and frees the server. */
void yt_server_destroy(struct yt_server* server);
/* Diagnostics (no counterpart in the paper): the worker treats its step number `at_tick`
 * (0 = the first; -1 = none) as failed, as if a CUDA call in it had returned an error,
 * without touching the device.  A failed step ends the server's service: the active
 * solves are freed and fail with YT_ERR_CUDA, pending requests fail, and later
 * yt_server_submit calls return YT_ERR_CUDA; yt_server_wait and yt_server_destroy still
 * return.  For testing that failure path. */
yt_status yt_server_fail_tick(struct yt_server* server, int64_t at_tick);

/* Host-only diagnostics: the global-matrix operands of the tensor-core kernels of an order
 * (2..7) as uploaded by a YT_BF16X3_F32ACC solver; kernel 0 = the local kernel (passes:
 * CK derivatives -- at order 7 the first derivative as two passes over its output rows
 * [0, 32) and [32, 56) --, volume chunks, face projections), 1 = the neighbour kernel
 * (lifting).
 * Each pass is an N x K matrix stored twice (bf16 hi parts, then lo parts) in the
 * K-major canonical layout of 8 x 8 core matrices: entry (n, k) at byte
 * (n/8)*16K + (k/8)*128 + (n%8)*16 + (k%8)*2.  `bytes` receives the size; pass out == NULL
 * to query it.  No counterpart in the paper. */
yt_status yt_tc_operands(int32_t order, int32_t kernel, unsigned char* out, int64_t* bytes);
/* Diagnostics: checks on the current device the integer-unit binary32 <-> binary64
 * conversions used by the reduced-precision kernels against the hardware conversions:
 * all 2^32 binary32 values (widening, exact; a subnormal input must give the signed
 * zero) and 2^28 binary64 values with one in eight a rounding tie (narrowing, round to
 * nearest even; a result the hardware rounds to a subnormal float counts as correct when
 * ours is the signed zero).  Writes the numbers of
 * mismatches; synchronous.  No counterpart in the paper. */
yt_status yt_selftest_conversions(int64_t* f2d_mismatches, int64_t* d2f_mismatches);
/* Host-only: reference matrices for an order without creating a solver (same meaning as
 * yt_solver_reference_matrix).  Runs no device code. */
yt_status yt_reference_matrix(int32_t order, const char* name, double* out, int64_t* count);

#ifdef __cplusplus
}
#endif
#endif /* YATETO_GB300_H */
