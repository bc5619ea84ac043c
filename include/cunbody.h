/*
 * cunbody.h - C ABI of libcunbody, softened direct-summation gravity on
 * NVIDIA GB300 (sm_103a).
 *
 * The library computes, for i-particles with positions x_i and
 * j-particles with positions x_j and masses m_j, the softened acceleration
 * of Eq. 1 (Section 1.1), with G = 1 and r_ij = r_j - r_i:
 *
 *     a_i   =  sum_j m_j (x_j - x_i) / (|x_j - x_i|^2 + eps2)^(3/2)
 *     phi_i = -sum_{j : x_j != x_i} m_j / (|x_j - x_i|^2 + eps2)^(1/2)
 *
 * The call shape follows the library routine of Section 3.1 (Figure
 * "structure of subroutine of our library": j positions and masses, i
 * positions, the squared softening eps2, the output accelerations, n_i and
 * n_j), with positions and masses packed into 16-byte records as in the
 * appendix driver (JDIM = 4: x, y, z, m).
 *
 * Conventions shared by every entry point:
 *  - Array arguments are DEVICE pointers owned by the caller unless the
 *    name says "host", in memory of the current device (kernels launch on
 *    the current device; the library does not check where a pointer lives). Particle arrays are float[n][4] records
 *    (x, y, z, m), 16-byte aligned (else CN_ERR_MISALIGNED); the 4th
 *    component of an i-record is ignored. The i and j arrays may be the
 *    same buffer. Outputs must not overlap inputs.
 *  - eps2 is the SQUARED softening length (the pipeline descriptions of the
 *    appendix add it to dx^2 + dy^2 + dz^2); it must be finite and >= 0.
 *  - A pair with |x_j - x_i|^2 + eps2 == 0 (eps2 = 0 and coincident points)
 *    contributes nothing. The potential skips every pair whose coordinate
 *    differences are all exactly zero, so the i = j self term is excluded.
 *    (Separations below about 1e-19, whose squares flush to zero in FP32,
 *    count as zero.)
 *  - n_i == 0 is a no-op; n_j == 0 writes zeros.
 *  - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *    default stream). Argument errors are detected on the host and returned
 *    before anything is launched. Results are valid after the stream is
 *    synchronised. cn_get_device_status reports errors detected inside a
 *    kernel (every wait inside a kernel is bounded in time).
 *  - Entry points without a `workspace` argument use a workspace owned by
 *    the library, kept per (device, stream) and grown on demand; growing it
 *    allocates, which is not allowed while `stream` is being captured into
 *    a CUDA graph (CN_ERR_WORKSPACE): make one call on that stream before
 *    capturing, or use the *_ws forms.
 *  - Thread safety: concurrent calls are safe on different streams.
 *  - Errors are returned as cn_status codes, with a message from
 *    cn_last_error_message (per thread). No C++ exception leaves the
 *    library: host memory exhausted inside it, or any other C++ runtime
 *    error, is CN_ERR_HOST.
 *  - Kernels are launched with programmatic stream serialization
 *    (programmatic dependent launch): a library kernel may be scheduled
 *    while the previous kernel of the stream is still running, and it waits
 *    for that kernel to complete before it touches global memory, so stream
 *    order holds for the data. A kernel of the caller's that follows a
 *    library call in the stream and is itself launched with that attribute
 *    must wait in the same way (cudaGridDependencySynchronize) before it
 *    reads the library's outputs.
 *  - Environment: CN_PDL=0 launches in plain stream order and CN_LOG=1
 *    prints one line per launch (variant, shape, grid, split tiles) to
 *    stderr (both read once per process); CN_FAULT_INJECT, a comma list of
 *    alloc, launch and capture, makes those host steps fail as if the CUDA
 *    call had failed, and hostmem makes the host-side building of a batch or
 *    list plan fail as if host memory were exhausted (CN_ERR_HOST) (read at
 *    every call; for testing error paths).
 */
#ifndef CUNBODY_H
#define CUNBODY_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define CN_API __attribute__((visibility("default")))
#else
#define CN_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; declared here so the header needs no CUDA headers. */
typedef struct CUstream_st *cn_stream;

typedef enum cn_status {
    CN_OK = 0,
    CN_ERR_INVALID_ARG = 1,        /* a size, pointer or eps2 is invalid                     */
    CN_ERR_MISALIGNED = 2,         /* a float[n][4] array is not 16-byte aligned             */
    CN_ERR_CUDA = 3,               /* a CUDA runtime call failed (see cn_last_error_message)  */
    CN_ERR_TIMEOUT = 4,            /* a kernel gave up waiting (reported by cn_get_device_status) */
    CN_ERR_UNSUPPORTED_DEVICE = 5, /* the current device is not sm_103 (GB300)               */
    CN_ERR_WORKSPACE = 6,          /* workspace too small, or allocation needed during capture */
    CN_ERR_HOST = 7                /* host-side failure inside the library: host memory exhausted
                                      or another C++ runtime error (no exception leaves the library) */
} cn_status;

/* Kernel variants, used by the workspace, tuning and autotuning calls. */
typedef enum cn_variant {
    CN_VARIANT_F32 = 0,        /* cn_force without potential      */
    CN_VARIANT_F32_POT = 1,    /* cn_force with potential         */
    CN_VARIANT_DD = 2,         /* cn_force_dd without potential   */
    CN_VARIANT_DD_POT = 3,     /* cn_force_dd with potential      */
    CN_VARIANT_ADJOINT = 4,    /* cn_force_adjoint                */
    CN_VARIANT_BATCHED = 5,    /* cn_force_batched                */
    CN_VARIANT_BATCHED_POT = 6, /* cn_force_batched with potential */
    CN_VARIANT_JERK = 7,        /* cn_force_jerk without potential */
    CN_VARIANT_JERK_POT = 8,    /* cn_force_jerk with potential    */
    CN_VARIANT_SYMMETRIC = 9,   /* cn_force_symmetric              */
    CN_VARIANT_F32_EPS_I = 10,  /* cn_force_eps_i without potential */
    CN_VARIANT_F32_EPS_I_POT = 11 /* cn_force_eps_i with potential */
} cn_variant;

/* Launch shape of the pair kernels. Zero in a field means "library default". */
typedef struct cn_tune {
    int32_t i_per_thread; /* i-particles held in registers per thread: 1, 2, 4 or 8              */
    int32_t threads;      /* threads per CTA: 64, 128 or 256                                      */
    int32_t j_tile;       /* j records per shared-memory stage: multiple of 16, 16 .. 4096        */
    int32_t stages;       /* shared-memory ring depth: 1 .. 8 (1: one tile in flight at a time)   */
    int32_t ctas_per_sm;  /* resident CTAs per SM to launch (0 = occupancy maximum)               */
    int32_t chunk_units;  /* 0 = static schedule (equal share per CTA); > 0 = dynamic queue chunks
                             of this many (i-tile x j-tile) units. Symmetric form: tile rows per
                             band (0 = one band while its slots fit in 2 GiB, else bands)       */
    int32_t j_lanes;      /* single-system FP32, per-i-softening, force-jerk and adjoint forms:
                             lanes sharing the thread's i-particles (1, 2, 4, ..., 32; needs
                             j_tile a multiple of 8 x j_lanes; i_per_thread up to 8 for the
                             plain FP32 forms, 1 or 2 for per-i softening, exactly 2 for the
                             force-jerk and adjoint forms); their partial sums are combined
                             by warp shuffles. Ignored (1) for calls with eps2 = 0
                             of the force-jerk and adjoint forms                                */
} cn_tune;

/* ------------------------------------------------------------------ force */

/*
 * Plain FP32 direct sum (Eq. 1, and the potential when pot_out != NULL).
 *   n_i, pos_i       : i-particles, float[n_i][4] (4th component ignored)
 *   n_j, pos_mass_j  : j-particles, float[n_j][4] (x, y, z, m)
 *   eps2             : squared softening (finite, >= 0)
 *   acc_out          : float[n_i][3] accelerations (written)
 *   pot_out          : float[n_i] potentials phi_i, or NULL
 * FP32 pair arithmetic with the MUFU inverse square root; each j-tile's
 * FP32 partial is folded into an FP32 running sum (the FORCE-LOOP of
 * Section 2.2.2, Eq. 2); partial sums of i-tiles split across CTAs are
 * merged in FP64 in a fixed order, so results are bitwise reproducible for
 * a given launch shape.
 */
CN_API cn_status cn_force(int64_t n_i, const float *pos_i, int64_t n_j, const float *pos_mass_j, float eps2,
                   float *acc_out, float *pot_out, cn_stream stream);

/* cn_force with a caller-owned workspace of ws_bytes >= cn_workspace_bytes(
 * pot_out ? CN_VARIANT_F32_POT : CN_VARIANT_F32, n_i, n_j), 256-byte
 * aligned. It needs no initialisation: each call clears the workspace's
 * control head (queue words and split-tile arrival counters) with one
 * cudaMemsetAsync on `stream` before the kernel. No allocation happens
 * inside this call. Calls sharing a workspace must not overlap in time on
 * the device. */
CN_API cn_status cn_force_ws(int64_t n_i, const float *pos_i, int64_t n_j, const float *pos_mass_j, float eps2,
                      float *acc_out, float *pot_out, void *workspace, size_t ws_bytes, cn_stream stream);

/*
 * Compensated ("split-precision") direct sum with FP64 outputs.
 *   acc_out : double[n_i][3]; pot_out : double[n_i] or NULL; other
 *   arguments as cn_force.
 * FP32 instructions only: the pair term is evaluated in FP32 with the
 * roundings that matter recovered (a fast two-sum for x_j - x_i, exact
 * squares and ordered two-sums for the softened squared distance, the MUFU
 * inverse square root corrected to first order by an FMA-formed residual,
 * the residuals of the mass and direction products); each term is added to
 * a (hi, lo) FP32 running sum with Knuth's TwoSum, and the sums of every
 * j-tile are folded into FP64. Partial sums of split i-tiles are merged in
 * FP64 in a fixed order. Per-particle relative error against an exact sum:
 * ~1e-9 on Plummer spheres, 1.6e-8 at worst on the N = 2^20 Hernquist
 * workload (the FP32 form: ~1e-6).
 * The wide accumulators of the GRAPE pipelines (Section 1.6) and the
 * FORCE-LOOP error analysis (Section 2.2.2) motivate the form.
 */
CN_API cn_status cn_force_dd(int64_t n_i, const float *pos_i, int64_t n_j, const float *pos_mass_j, float eps2,
                      double *acc_out, double *pot_out, cn_stream stream);

/* cn_force_dd with a caller-owned workspace (same rules as cn_force_ws,
 * sized by CN_VARIANT_DD / CN_VARIANT_DD_POT). */
CN_API cn_status cn_force_dd_ws(int64_t n_i, const float *pos_i, int64_t n_j, const float *pos_mass_j, float eps2,
                         double *acc_out, double *pot_out, void *workspace, size_t ws_bytes, cn_stream stream);

/* Workspace bytes that a call of `variant` with these sizes needs under the
 * launch shape currently selected for them (see cn_tune_get). For
 * CN_VARIANT_ADJOINT pass n_i = n_j = n. Returns 0 for invalid input. */
CN_API size_t cn_workspace_bytes(int variant, int64_t n_i, int64_t n_j);

/*
 * cn_force for callers that cannot allocate device memory. The paper has no
 * counterpart; it exists because some callers may not call cudaMalloc at
 * all - a host application whose own memory manager owns every device
 * allocation, or a latency-bound loop that cannot afford the device-wide
 * synchronisation that cudaMalloc and cudaFree may imply - while cn_force
 * grows a library workspace on demand and cn_force_ws needs a buffer from
 * the caller.
 *   Arguments, results and errors as cn_force; nothing is allocated.
 *   Scratch: a fixed 32 MiB array in the library's device image. A problem
 *   whose launch shape needs more scratch than that (see
 *   cn_workspace_bytes) is rejected with CN_ERR_WORKSPACE before anything
 *   runs.
 *   Set-up: the library's first call of any entry point on a device (this
 *   one or another) sets that device up, which looks up the array's device
 *   address and, under CUDA's lazy module loading, loads the library's
 *   device code there - allocating the 32 MiB, which the GPU then holds
 *   until the process exits. Likewise the first launch of each kernel in a
 *   process loads that kernel's code. So make one cn_force call with the
 *   same sizes (or set CUDA_MODULE_LOADING=EAGER) on each device before the
 *   region where allocation is not allowed, and before capturing any
 *   stream; after that this call allocates nothing.
 *   Every call uses the same array: calls that overlap on the GPU (other
 *   streams, other host threads) race and corrupt each other's results, so
 *   serialise them. Each call clears the part that must start at zero.
 */
CN_API cn_status cn_force_noalloc(int64_t n_i, const float *pos_i, int64_t n_j, const float *pos_mass_j, float eps2,
                                  float *acc_out, float *pot_out, cn_stream stream);

/*
 * cn_force with a softening per i-particle, as in the appendix's force
 * pipeline, whose i record is (x, y, z, eps2) (IDIM = 4): every pair (i, j)
 * uses the squared softening eps2_i of its i-particle.
 *   pos_eps_i  : float[n_i][4] device records (x, y, z, eps2_i), 16-byte
 *                aligned; each eps2_i finite and >= 0 (not checked: the
 *                values are on the device). A pair with s = 0 (eps2_i = 0
 *                and coincident points) contributes nothing.
 *   pos_mass_j, acc_out, pot_out, stream: as cn_force.
 * Same kernels and launch shapes as cn_force (tuned under
 * CN_VARIANT_F32_EPS_I / _POT), always with the s = 0 guard; with every
 * eps2_i equal to one value the results are bitwise those of cn_force.
 * Errors as cn_force.
 */
CN_API cn_status cn_force_eps_i(int64_t n_i, const float *pos_eps_i, int64_t n_j, const float *pos_mass_j,
                                float *acc_out, float *pot_out, cn_stream stream);

/*
 * Accelerations of Eq. 1 for n particles under each other's gravity (i set
 * = j set), evaluating every unordered pair once (Newton's third law: the
 * pair term is added to one particle and subtracted, with the other mass,
 * from the other). Not in the paper, whose kernel evaluates every ordered
 * pair: 16 FP32 lane operations and one MUFU per unordered pair plus a warp
 * reduce-scatter of the j-side sums, against 2 x 12 for the two ordered
 * pairs. The j-side sums of each tile pair and the i-side sums of each
 * (CTA, tile row) segment are merged per particle in FP64 in a fixed order
 * (bitwise reproducible for a given launch shape); accuracy as cn_force.
 * It pays off from about N = 24576 on a GB300 (1.15x cn_force at 24576,
 * 1.29x at 131072); at N = 16384 the two take the same time and below it
 * cn_force is faster (about 1.9x at 8192).
 *   pos_mass : float[n][4] device records (x, y, z, m), 16-byte aligned
 *   eps2     : softening squared, finite and >= 0 (0: coincident pairs
 *              contribute nothing)
 *   acc_out  : float[n][3] device, 4-byte aligned, must not overlap pos_mass
 *   pot_out  : float[n] potentials or NULL (the pair's -m r to both sides,
 *              skipping pairs at exactly zero separation, as cn_force)
 * Asynchronous on `stream`; n == 0 is a no-op. Errors: CN_ERR_INVALID_ARG
 * (n < 0, bad eps2, NULL or overlapping buffers, a tune with j_lanes),
 * CN_ERR_MISALIGNED, CN_ERR_CUDA (launch), CN_ERR_WORKSPACE (below).
 * Uses a library workspace of j-side slots, 16 N^2 / B bytes for tiles of
 * B particles (134 MB at N = 131072 with the default 2048-particle tiles,
 * half of it written), plus the i-side segments (32 B per particle of a
 * tile per CTA and row), while the slots fit in 2 GiB; above, the tile rows
 * are processed in bands of w rows (about 16 w N + 32 N bytes, w chosen to
 * fit 2 GiB, or set by the tune's chunk_units), one kernel and one merge
 * per band. A banded launch cuts the rows into other segments than a
 * one-band launch, so the two agree to FP32 rounding of the segment sums,
 * not bitwise. CN_ERR_WORKSPACE when even one band cannot be held.
 */
CN_API cn_status cn_force_symmetric(int64_t n, const float *pos_mass, float eps2, float *acc_out, float *pot_out,
                                    cn_stream stream);

/* ------------------------------------------------------------------ batched */

/* An ensemble of independent systems ("clusters") stored back to back:
 * cluster c owns records offsets[c] .. offsets[c+1]-1 and softening
 * eps2[c]; every cluster is its own i set and j set. A plan holds the
 * (cluster, i-tile, j-tile) unit table in device memory; it is built once
 * per ensemble shape on the current device. This is the many-small-systems
 * use of Section 4.4 (groups of particles sharing one interaction list in
 * the modified tree algorithm) in a single persistent launch. */
typedef struct cn_batch_plan cn_batch_plan;

/* offsets_host: int64[n_clusters + 1], non-decreasing, offsets_host[0] == 0;
 * eps2_host: float[n_clusters]; tune: launch shape or NULL (default or the
 * shape stored by cn_tune_set for CN_VARIANT_BATCHED); with_potential:
 * nonzero to reserve the potential form. Allocates device memory. */
CN_API cn_status cn_batch_plan_create(int32_t n_clusters, const int64_t *offsets_host, const float *eps2_host,
                               const cn_tune *tune, int with_potential, cn_batch_plan **plan_out);
CN_API cn_status cn_batch_plan_destroy(cn_batch_plan *plan);
/* Workspace bytes a cn_force_batched call on this plan needs. */
CN_API size_t cn_batch_plan_workspace_bytes(const cn_batch_plan *plan);
/* Number of particles (offsets[n_clusters]) and pair interactions
 * (sum_c N_c^2) the plan covers; either pointer may be NULL. */
CN_API cn_status cn_batch_plan_info(const cn_batch_plan *plan, int64_t *n_total, double *pairs);

/*
 * One persistent launch over all clusters of `plan`.
 *   pos_mass  : float[n_total][4] records of all clusters
 *   acc_out   : float[n_total][3]; pot_out : float[n_total] or NULL
 *   workspace : caller-owned, >= cn_batch_plan_workspace_bytes(plan) bytes,
 *               256-byte aligned, no initialisation needed (its control
 *               head is cleared on `stream` before the kernel); NULL to use
 *               the library workspace of `stream`.
 * No allocation happens when a workspace is passed, so the call can be
 * captured into a CUDA graph (see cn_batch_plan_capture).
 */
CN_API cn_status cn_force_batched(const cn_batch_plan *plan, const float *pos_mass, float *acc_out, float *pot_out,
                           void *workspace, size_t ws_bytes, cn_stream stream);

/* Captures cn_force_batched with these arguments into a CUDA graph owned by
 * the plan (replacing any earlier one); cn_batch_plan_launch replays it. */
CN_API cn_status cn_batch_plan_capture(cn_batch_plan *plan, const float *pos_mass, float *acc_out, float *pot_out,
                                void *workspace, size_t ws_bytes, cn_stream stream);
CN_API cn_status cn_batch_plan_launch(const cn_batch_plan *plan, cn_stream stream);

/* Interaction lists: the use of the O(N^2) engine inside the modified tree
 * algorithm (Section 4.4), where a group of neighbouring i-particles shares
 * one list of j records (particles and tree-node pseudo-particles, each an
 * (x, y, z, m) record) gathered by the tree code. Group g evaluates the
 * i-particles i_offsets[g] .. i_offsets[g+1]-1 of pos_i against the j
 * records j_begin[g] .. j_begin[g] + j_count[g] - 1 of pos_mass_j with
 * softening eps2[g]; lists may overlap or be shared. The plan (a unit table
 * in device memory) is built once per list structure on the current device.
 *   i_offsets_host : int64[n_groups + 1], non-decreasing, i_offsets[0] == 0
 *   j_begin_host, j_count_host : int64[n_groups], >= 0
 *   eps2_host      : float[n_groups]
 * Destroy with cn_batch_plan_destroy; workspace size from
 * cn_batch_plan_workspace_bytes; cn_batch_plan_info reports the number of
 * i-particles and the pair count sum_g n_i,g n_j,g. */
CN_API cn_status cn_list_plan_create(int32_t n_groups, const int64_t *i_offsets_host, const int64_t *j_begin_host,
                                     const int64_t *j_count_host, const float *eps2_host, const cn_tune *tune,
                                     int with_potential, cn_batch_plan **plan_out);

/* Interaction lists as index arrays: the form a tree code's walk produces
 * (Section 4.4), where a list names particles and tree nodes of one source
 * array instead of holding copies of their records. Group g evaluates its
 * i-particles against the records pos_mass_j[j_index[e]] for the entries
 * e = j_begin[g] .. j_begin[g] + j_count[g] - 1 of j_index, in that order;
 * entries may repeat and lists may share or overlap entries. The kernel
 * gathers each j-tile's records into shared memory itself (no copy of the
 * lists is written to device memory).
 *   i_offsets_host, j_begin_host, j_count_host, eps2_host : as for
 *                    cn_list_plan_create, with j ranges counting entries
 *   j_index_host   : int32[n_index] (NULL only when n_index == 0), copied
 *                    into the plan; the host array is not kept
 *   n_src          : number of records of the source array that
 *                    cn_force_lists will read (at most INT32_MAX)
 * Every entry a group with i-particles reaches must lie in 0 .. n_src - 1,
 * and every list inside 0 .. n_index - 1: checked here, on the host;
 * CN_ERR_INVALID_ARG otherwise. The plan runs with cn_force_lists (and
 * cn_list_plan_capture), pos_mass_j then being the n_src source records. A
 * plan made by cn_list_plan_create with the same arguments and the same
 * launch shape (tune), run on the records pos_mass_j[j_index[e]] laid out
 * in entry order, gives the same bits (the same records in the same order).
 * Without a tune the two may differ in shape: where the fit lands on K = 8
 * with lane groups, a gathering plan takes K = 4 with half of them (its
 * threads also stage the records). */
CN_API cn_status cn_list_plan_create_indexed(int32_t n_groups, const int64_t *i_offsets_host,
                                             const int64_t *j_begin_host, const int64_t *j_count_host,
                                             const float *eps2_host, const int32_t *j_index_host, int64_t n_index,
                                             int64_t n_src, const cn_tune *tune, int with_potential,
                                             cn_batch_plan **plan_out);

/* One persistent launch over all groups of a list plan.
 *   pos_i      : float[n_i][4] (n_i = i_offsets[n_groups]; 4th component ignored)
 *   pos_mass_j : float[*][4] lists, long enough for every group's range
 *                (gathering plans: the n_src source records)
 *   acc_out    : float[n_i][3]; pot_out : float[n_i] or NULL (groups with an
 *                empty list get zeros)
 *   workspace  : as for cn_force_batched. */
CN_API cn_status cn_force_lists(const cn_batch_plan *plan, const float *pos_i, const float *pos_mass_j,
                                float *acc_out, float *pot_out, void *workspace, size_t ws_bytes, cn_stream stream);
/* cn_batch_plan_capture for list plans (cn_batch_plan_launch replays it). */
CN_API cn_status cn_list_plan_capture(cn_batch_plan *plan, const float *pos_i, const float *pos_mass_j,
                                      float *acc_out, float *pot_out, void *workspace, size_t ws_bytes,
                                      cn_stream stream);

/* ------------------------------------------------------------------ adjoint */

/*
 * Gradient of L = sum_i w_i . a_i (i set = j set = all n particles) with
 * respect to every position and mass, in one O(n^2) pass:
 *   dL/dx_k = sum_p [ g u - 3 h (d . u) d ],  dL/dm_k = -sum_p g (w_p . d)
 * with d = x_p - x_k, s = |d|^2 + eps2, g = s^-3/2, h = s^-5/2,
 * u = m_k w_p - m_p w_k. The paper has no adjoint; this is the derivative
 * of Eq. 1.
 *   pos_mass  : float[n][4]; w : float[n][3] (any 4-byte alignment)
 *   grad_pos  : float[n][3]; grad_mass : float[n] (both written)
 * FP32 pair arithmetic, per-tile FP32 partials, FP64 merge of split tiles.
 */
CN_API cn_status cn_force_adjoint(int64_t n, const float *pos_mass, float eps2, const float *w, float *grad_pos,
                           float *grad_mass, cn_stream stream);

/* ------------------------------------------------------------------ force, jerk, potential */

/*
 * The outputs of the force-jerk-potential pipeline description of the
 * appendix (what a Hermite integrator needs each step): for i-particles with
 * positions x_i and velocities v_i and j-particles (x_j, m_j, v_j),
 *   a_i   =  sum_j m_j d / s^(3/2)
 *   j_i   =  sum_j m_j [ w / s^(3/2) - 3 (d . w) d / s^(5/2) ]   (= d a_i / dt)
 *   phi_i = -sum_{j : d != 0} m_j / s^(1/2)
 * with d = x_j - x_i, w = v_j - v_i, s = |d|^2 + eps2.
 *   pos_i, vel_i        : float[n_i][4] (4th components ignored)
 *   pos_mass_j, vel_j   : float[n_j][4] ((x, y, z, m) and (vx, vy, vz, -))
 *   acc_out, jerk_out   : float[n_i][3]; pot_out : float[n_i] or NULL
 * All four record arrays 16-byte aligned. FP32 pair arithmetic (27 FP32
 * instructions and one MUFU inverse square root per pair), per-tile FP32
 * partials folded into running sums, FP64 merge of split tiles. The
 * appendix hard-wires eps2 = 1/256^2; here it is an argument.
 */
CN_API cn_status cn_force_jerk(int64_t n_i, const float *pos_i, const float *vel_i, int64_t n_j,
                               const float *pos_mass_j, const float *vel_j, float eps2, float *acc_out,
                               float *jerk_out, float *pot_out, cn_stream stream);

/* ------------------------------------------------------------------ potential energy */

/* W = 1/2 sum_i m_i phi_i accumulated in FP64 in a fixed order.
 * pos_mass: float[n][4] (masses in the 4th component); pot: float[n]
 * (cn_potential_energy) or double[n] (cn_potential_energy_dd);
 * w_out: ONE double in device memory (written). */
CN_API cn_status cn_potential_energy(int64_t n, const float *pos_mass, const float *pot, double *w_out, cn_stream stream);
CN_API cn_status cn_potential_energy_dd(int64_t n, const float *pos_mass, const double *pot, double *w_out,
                                 cn_stream stream);

/* ------------------------------------------------------------------ host-memory forms */

/* cn_force on HOST buffers: copies pos_i and pos_mass_j to the device,
 * evaluates, copies acc (and pot) back and returns when they are in host
 * memory. Uses device buffers kept by the library per (device, stream).
 * Pinned host memory gives the fastest copies. */
CN_API cn_status cn_force_host(int64_t n_i, const float *pos_i_host, int64_t n_j, const float *pos_mass_j_host, float eps2,
                        float *acc_host, float *pot_host, cn_stream stream);

/* The library routine exactly as Section 3.1 states it: FP64 host arrays
 * xj[nj][3], mj[nj], xi[ni][3], the squared softening eps2 and the output
 * a[ni][3]. Values are rounded to FP32 records (as the appendix driver
 * packs them), evaluated with cn_force on the legacy default stream, and
 * widened back. Synchronous. */
CN_API cn_status cn_force_host_f64(const double *xj, const double *mj, const double *xi, double eps2, double *a, int ni,
                            int nj);

/* ------------------------------------------------------------------ tuning */

/* Launch shape that calls of `variant` with these sizes will use on the
 * current device: an entry set by cn_tune_set / cn_autotune for the size
 * class (ceil(log2 n_i), ceil(log2 n_j)), else the built-in heuristic. */
CN_API cn_status cn_tune_get(int variant, int64_t n_i, int64_t n_j, cn_tune *out);
/* Stores (tune != NULL) or clears (tune == NULL) the shape for the size class. */
CN_API cn_status cn_tune_set(int variant, int64_t n_i, int64_t n_j, const cn_tune *tune);

/*
 * Persisted tuning table (the paper has no counterpart; tuning is this
 * library's own state). cn_tune_save writes every entry stored for the
 * current device (by cn_tune_set or the autotuners) to `path` as JSON:
 *   {"format": "cunbody-tune-1", "device": "<name>", "arch": "sm_103",
 *    "sms": <multiprocessors>, "entries": [{"variant": "f32", "n_i_class": 17,
 *    "n_j_class": 17, "i_per_thread": 8, ...}, ...]}
 * where a size class is ceil(log2 n). Overwrites the file; CN_ERR_INVALID_ARG
 * if it cannot be written.
 * cn_tune_load reads such a file and stores its entries for the current
 * device, replacing entries of the same variant and size classes. The whole
 * file is parsed and checked first (CN_ERR_INVALID_ARG for a missing or
 * malformed file or an invalid entry, with nothing stored); a file written
 * on a device with another name, arch or multiprocessor count is refused
 * with CN_ERR_UNSUPPORTED_DEVICE. *n_loaded (if not NULL) receives the
 * number of entries stored. Host-side only; no device work.
 */
CN_API cn_status cn_tune_save(const char *path);
CN_API cn_status cn_tune_load(const char *path, int32_t *n_loaded);

/*
 * Times every candidate launch shape for `variant` on these inputs (CUDA
 * events on `stream`, best of `reps`), stores the fastest with cn_tune_set
 * and returns it in best_out. Outputs are overwritten; synchronises
 * `stream`. For the DD variants acc_out/pot_out point to double arrays,
 * for the F32 variants to float arrays. Not for CN_VARIANT_ADJOINT or the
 * batched variants (see cn_autotune_batched).
 */
CN_API cn_status cn_autotune(int variant, int64_t n_i, const float *pos_i, int64_t n_j, const float *pos_mass_j,
                      float eps2, void *acc_out, void *pot_out, int reps, cn_stream stream, cn_tune *best_out);

/* Times candidate shapes for a batched ensemble (building a plan for each),
 * returns the fastest in best_out and stores it for CN_VARIANT_BATCHED /
 * CN_VARIANT_BATCHED_POT keyed by (number of clusters, total particles). */
CN_API cn_status cn_autotune_batched(int32_t n_clusters, const int64_t *offsets_host, const float *eps2_host,
                              const float *pos_mass, float *acc_out, float *pot_out, int reps, cn_stream stream,
                              cn_tune *best_out);

/* ------------------------------------------------------------------ status, probes */

/* Synchronises `stream` and reports CN_ERR_TIMEOUT if any kernel of this
 * library on the current device flagged a timed-out wait since the last
 * call (the flag is then cleared and library workspaces are re-zeroed), or
 * CN_ERR_CUDA if the synchronisation failed. */
CN_API cn_status cn_get_device_status(cn_stream stream);

/* Sets the bound on every in-kernel wait, in nanoseconds (default 2e9);
 * 0 restores the default. Applies to launches made after the call. */
CN_API cn_status cn_set_wait_limit_ns(uint64_t ns);

/* Launches one kernel that waits on a shared-memory barrier which nothing
 * completes, bounded by the current wait limit: the kernel then flags a
 * timeout and returns. Lets a test exercise the timeout path without a
 * hang; follow with cn_get_device_status. */
CN_API cn_status cn_debug_timeout_probe(cn_stream stream);

/* Measured issue rates of the current device (one probe kernel each):
 *   out[0] FP32 FFMA lane operations per second,
 *   out[1] MUFU inverse square roots per second,
 *   out[2] pair-equivalent rate of a loop of 12 FP32 + 1 MUFU per pair,
 *   out[3] mean SM clock during the probes in MHz,
 *   out[4] number of SMs.
 * Synchronises `stream`. */
CN_API cn_status cn_probe_peaks(cn_stream stream, double *out5);

CN_API const char *cn_status_string(cn_status status);
/* Detail of the last error on the calling thread (empty if none). */
CN_API const char *cn_last_error_message(void);
/* Library version string. */
CN_API const char *cn_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CUNBODY_H */
