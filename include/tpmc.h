/*
 * tpmc.h -- C ABI of the GB300 test-particle Monte Carlo (TPMC) library.
 *
 * The library computes the free-molecular force, torque and drag coefficient
 * of a triangulated body by the method of Parham & Barba, "Finding the Force
 * -- Consistent Particle Seeding for Satellite Aerodynamics" (arXiv 1312.3691):
 *
 *   1. free-stream particles are seeded on a spherical control volume (CV)
 *      with the number flux of Eq. 10, the latitude law g(phi|S) of Eq. 11,
 *      the velocity component laws of Eq. 14a-c, and the Rodrigues rotation
 *      of Eq. 15 into body coordinates (§III.A);
 *   2. each particle is ray traced to its closest hit on the surface, re-emitted
 *      by the gas-surface interaction model and traced again until it leaves
 *      (multiple reflections and self-shadowing, §II.A);
 *   3. the momentum differences, scaled by the particle weight Gamma/N times
 *      the molecular mass (§II.A), sum to the force; C_D follows Eq. 1.
 *
 * Conventions for every entry point:
 *   - every call returns a tpmc_status; nothing aborts or throws across the ABI;
 *   - pointers named h_* or documented "host" are host memory, d_* are device
 *     memory of the context's GPU; the caller owns every buffer it passes;
 *   - inputs are copied; meshes and their BVHs are owned by the context until
 *     tpmc_mesh_unload or tpmc_destroy;
 *   - a failed call leaves the context usable and sets tpmc_last_error();
 *   - calls on one context are serialised by an internal mutex (thread safe);
 *     GPU work runs on the context's stream (tpmc_set_stream).
 *
 * Units: SI (m, s, kg, K, N, N m).  Velocities inside the library are in
 * units of the most probable thermal speed c_mp = sqrt(2 k_B T_inf / m).
 */
#ifndef TPMC_H
#define TPMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TPMC_OK = 0,
  TPMC_EINVAL = 1,     /* invalid argument (non-finite, out of range, bad mesh) */
  TPMC_ENOMEM = 2,     /* device memory or the context's memory budget exhausted */
  TPMC_EBUSY = 3,      /* serving queue full: retry after a poll */
  TPMC_ETIMEOUT = 4,   /* tpmc_poll: the query has not finished within the timeout */
  TPMC_ECUDA = 5,      /* a CUDA runtime call failed (message in tpmc_last_error) */
  TPMC_ENOTFOUND = 6   /* unknown mesh id or query id */
} tpmc_status;

typedef struct tpmc_ctx tpmc_ctx;
typedef uint32_t tpmc_mesh_id;
typedef uint64_t tpmc_query_id;

/* Arithmetic of the per-particle path.  FP32: seeding, traversal, intersection
 * and re-emission in float; FP64 only for the flux normalisation (set-up) and
 * the final force/C_D reduction.  FP64: everything in double. */
enum { TPMC_FP32 = 0, TPMC_FP64 = 1 };

/* Control volume on which test particles are seeded (tpmc_params.cv_kind).
 *   TPMC_CV_SPHERE       the paper's consistent seeding on a sphere (§III.A:
 *                        Eq. 10 flux, Eq. 11 latitude, Eq. 14a-c velocity,
 *                        Eq. 15 rotation).  The default.
 *   TPMC_CV_BOX_FLUX     rectangular CV (§I, §III.A; the ANGARA scheme):
 *                        uniform points on the six faces, face f taking the
 *                        particle ids [floor(N C_f), floor(N C_{f+1})), C_f
 *                        the cumulative share of the flat-plate number flux
 *                        A_f n c G(s_f); inward normal speed from the
 *                        flux-weighted law of Eq. 14a at s_f = S Vhat.n_in.
 *                        Kinetically consistent: same expectation as the sphere.
 *   TPMC_CV_BOX_MAXWELL  the same faces and counts, but the inward normal speed
 *                        drawn from the free-stream Maxwellian restricted to
 *                        entering velocities (no flux factor): the
 *                        inconsistent seeding whose incidence-dependent bias
 *                        the paper reports.
 * Faces are ordered +x, -x, +y, -y, +z, -z (x_a = box_hi[a], then box_lo[a]).
 * Both box kinds use the same Philox draws as the sphere: the top 23 bits of
 * block 0's four words give the two face coordinates, the normal speed and
 * the tangential radius; 23 of their low bits give the tangential angle. */
enum { TPMC_CV_SPHERE = 0, TPMC_CV_BOX_FLUX = 1, TPMC_CV_BOX_MAXWELL = 2 };

/* Gas-surface interaction (tpmc_params.gsi_model).
 *   TPMC_GSI_MAXWELL  the paper's model (§II.A): a fraction eps_diffuse of the
 *                     hits re-emitted diffusely from the flux-weighted
 *                     half-range Maxwellian at T_W, the rest specularly.  The
 *                     default.
 *   TPMC_GSI_CLL      Cercignani-Lampis-Lord (Lord's sampling of the CL
 *                     kernel; not in the paper): normal-energy accommodation
 *                     alpha_n and tangential-momentum accommodation sigma_t,
 *                     both in [0, 1].  1, 1 is the diffuse law; 0, 0 is
 *                     specular reflection.  Uses the same Philox block per
 *                     bounce as the Maxwell model. */
enum { TPMC_GSI_MAXWELL = 0, TPMC_GSI_CLL = 1 };

/* One free-molecular query (§II.A; §III.C; Table 1 of the paper). */
typedef struct {
  double n;             /* free-stream number density, 1/m^3 (> 0)                      */
  double T_inf;         /* free-stream temperature, K (> 0)                             */
  double m;             /* molecular mass, kg (> 0)                                     */
  double V;             /* bulk speed, m/s (> 0); S = V / c_mp is derived, never passed */
  double dir[3];        /* flow direction in body coordinates (normalised by the library) */
  double T_W;           /* wall temperature, K (> 0)                                    */
  double eps_diffuse;   /* Maxwell accommodation: fraction re-emitted diffusely, [0,1]  */
  double A_ref;         /* C_D reference area, m^2 (> 0)                                */
  double ref_point[3];  /* torque reference point, m                                    */
  double r_cv;          /* CV radius, m; <= 0: 1.05 x the mesh's bounding radius       */
  double center[3];     /* CV centre, m (ignored when r_cv <= 0: bounding-sphere centre) */
  uint32_t max_bounces; /* hits per particle before it is stopped, 1 to 2^24-1, e.g. 64 */
  uint32_t precision;   /* TPMC_FP32 or TPMC_FP64                                       */
  uint64_t seed;        /* Philox key                                                   */
  uint32_t stream_id;   /* Philox counter word 2 (distinguishes runs sharing a seed)   */
  uint32_t want_panels; /* 1: keep per-triangle loads for tpmc_panels                   */
  uint32_t cv_kind;     /* TPMC_CV_SPHERE (0, default), TPMC_CV_BOX_FLUX, TPMC_CV_BOX_MAXWELL */
  uint32_t pad_cv;      /* must be 0                                                    */
  double box_lo[3];     /* box CV corners, body frame, m (box kinds only): the mesh must */
  double box_hi[3];     /* lie strictly inside; r_cv and center are then ignored         */
  double l_ref;         /* moment reference length, m, for CM (<= 0: 1 m), e.g. the chord c
                           of §III.D.1 with ref_point at c/4                               */
  uint32_t gsi_model;   /* TPMC_GSI_MAXWELL (0, default) or TPMC_GSI_CLL                 */
  uint32_t pad_gsi;     /* must be 0                                                    */
  double alpha_n;       /* CLL normal-energy accommodation, [0, 1]                      */
  double sigma_t;       /* CLL tangential-momentum accommodation, [0, 1]                */
} tpmc_params;

/* Result of one query.  force/torque in N and N m; CD = force . Vhat / (q_inf A_ref). */
typedef struct {
  double force[3], torque[3];
  double CD, CD_sigma;          /* C_D and its Monte Carlo standard error               */
  double CF[3];                 /* force / (q_inf A_ref), body axes                     */
  double CM[3];                 /* torque about ref_point / (q_inf A_ref l_ref), body axes;
                                   with A_ref = 1 m^2, CM is the area-scaled moment
                                   coefficient M / (q_inf c) of §III.D.1               */
  double S, S_W;                /* speed ratios V/c_mp and V/c_W                        */
  double gamma;                 /* molecules per second entering the CV (Eq. 10 for the
                                   sphere; sum of the faces' flat-plate fluxes for a box) */
  double weight;                /* molecules per second per simulated particle (Gamma/N) */
  double q_inf;                 /* dynamic pressure n m V^2 / 2, Pa                     */
  double c_mp;                  /* most probable thermal speed, m/s                     */
  double r_cv, center[3];       /* control volume used (box: r_cv = 0, centre of the box) */
  double fixed_quantum;         /* value of one unit of the int64 sums (c_mp units)     */
  int64_t sum_dv_q[3];          /* sum over hits of (v_in - v_out), fixed point         */
  int64_t sum_rdv_q[3];         /* sum over hits of (r_hit - ref) x (v_in - v_out)      */
  uint64_t n_particles, n_hits, n_hit_particles, n_truncated;
  uint64_t n_node_visits, n_tri_tests; /* traversal work (counted when enabled)         */
  tpmc_query_id query_id;       /* handle for tpmc_panels (want_panels = 1)             */
  double ms;                    /* wall time of the call or, when served, latency       */
  int32_t status;               /* tpmc_status of this query                            */
  int32_t pad_;
} tpmc_result;

/* Per-particle records for verification (host buffers, each may be NULL). */
typedef struct {
  double* pos;          /* [N][3] seeded position, body frame, m                        */
  double* vel;          /* [N][3] seeded velocity, c_mp units                           */
  double* dv;           /* [N][3] sum over the particle's hits of (v_in - v_out)        */
  uint32_t* n_hits;     /* [N] hits of the particle                                     */
  uint32_t* truncated;  /* [N] 1 when stopped at max_bounces                            */
  uint32_t* tri;        /* [N][K] triangle index of hit b (b < K), 0xFFFFFFFF after     */
  uint32_t K;           /* hits recorded per particle (<= 64)                           */
} tpmc_records;

typedef struct {
  uint32_t n_tri, n_vert, n_nodes, depth;
  uint32_t n_skipped;           /* zero-area triangles (never hit)                      */
  uint32_t leaf_max;            /* largest leaf                                          */
  double bound_center[3], bound_radius;
  uint64_t device_bytes;
  uint32_t n_refs;              /* triangle references in the leaves: spatial splits    */
                                /* put parts of some triangles in several leaves         */
  uint32_t n_exposed;           /* triangle sides with the whole mesh behind them: a    */
                                /* particle re-emitted from one is not traced further    */
  uint32_t bvh_width;           /* children per BVH node: 2 (binary, 64-byte nodes) or  */
                                /* 4 / 8 (compressed wide nodes of 80 bytes)             */
  uint32_t node_bytes;          /* bytes the trace kernel reads per node visit           */
} tpmc_mesh_stats;

/* Launch schedule of the trace kernel (chosen by tpmc_tune or set by hand). */
typedef struct {
  uint32_t block;               /* threads per block (multiple of 32)                   */
  uint32_t blocks_per_sm;       /* resident blocks per SM (grid = SMs x this)           */
  uint32_t chunk;               /* particle ids a warp takes per fetch (0: automatic)   */
  uint32_t smem_nodes;          /* BVH nodes staged in shared memory                    */
  uint32_t refill_at;           /* finished lanes that end a traversal round (0: 16)    */
  uint32_t bvh_leaf;            /* largest BVH leaf for later tpmc_mesh_load (0: 4)     */
  uint32_t bvh_width;           /* children per BVH node for later tpmc_mesh_load: 2, 4  */
                                /* or 8 (0: the default, or what tpmc_tune chose for     */
                                /* meshes of that size class)                            */
} tpmc_launch;

/* ---- context ------------------------------------------------------------ */

/* Creates a context on CUDA device `device` that may hold at most
 * mem_budget_bytes of device memory (0: 90 % of the free memory).
 * Errors: EINVAL (bad device), ECUDA. */
tpmc_status tpmc_create(int device, size_t mem_budget_bytes, tpmc_ctx** out);

/* Waits for the context's work, frees everything it owns. NULL is a no-op. */
tpmc_status tpmc_destroy(tpmc_ctx* ctx);

/* Makes later GPU work run on `cuda_stream` (a cudaStream_t; NULL = the
 * context's own stream).  The caller keeps the stream alive. */
tpmc_status tpmc_set_stream(tpmc_ctx* ctx, void* cuda_stream);

/* Thread-local message describing the last failure on this thread. */
const char* tpmc_last_error(const tpmc_ctx* ctx);

/* Device memory of the context: *used, the bytes it holds through its own
 * allocations (meshes and their BVHs, scratch, panel buffers, serving slots),
 * *budget, the limit set at creation, and *n_allocs, the number of device
 * allocations it has made since creation.  Any pointer may be NULL. */
tpmc_status tpmc_memory_info(tpmc_ctx* ctx, size_t* used, size_t* budget, uint64_t* n_allocs);

/* Enables (1) or disables (0) the traversal counters n_node_visits and
 * n_tri_tests in later results. */
tpmc_status tpmc_set_counters(tpmc_ctx* ctx, int enable);

/* ---- geometry (§II.A: "satellite surfaces are represented by a triangulation") */

/* Copies the mesh (xyz: host [n_vert][3] m; tri: host [n_tri][3] vertex
 * indices), builds its bounding-volume hierarchy on the host (surface-area
 * heuristic with spatial splits: at most 1.5 references per triangle) and
 * keeps both on the device.  Triangles are two-sided; the winding fixes the sign of the
 * geometric normal used for panel pressure.  Zero-area triangles are kept in
 * the numbering but never hit (counted in tpmc_mesh_stats.n_skipped).
 * Errors: EINVAL (n_vert = 0 with n_tri > 0, index out of range, non-finite
 * coordinate, n_tri > 2^24), ENOMEM. */
tpmc_status tpmc_mesh_load(tpmc_ctx* ctx, const double* xyz, uint32_t n_vert, const uint32_t* tri,
                           uint32_t n_tri, tpmc_mesh_id* out);
tpmc_status tpmc_mesh_unload(tpmc_ctx* ctx, tpmc_mesh_id mesh);
tpmc_status tpmc_mesh_info(tpmc_ctx* ctx, tpmc_mesh_id mesh, tpmc_mesh_stats* out);

/* ---- the hot path ------------------------------------------------------- */

/* Traces N particles of one query and returns its result (host), blocking.
 * Particle ids 0..N-1 index the Philox counters, so the result depends only
 * on (mesh, params, N), never on the schedule.
 * Errors: EINVAL (non-finite or non-positive n, T_inf, m, V, T_W, A_ref; eps
 * outside [0,1]; zero dir; max_bounces = 0 or above 2^24 - 1; N = 0 or
 * N > 2^34; a mesh vertex outside the given CV; a fixed-point overflow bound
 * that no quantum >= 2^-40 satisfies), ENOTFOUND, ENOMEM, ECUDA. */
tpmc_status tpmc_trace(tpmc_ctx* ctx, tpmc_mesh_id mesh, const tpmc_params* params, uint64_t N,
                       tpmc_result* out);

/* Per-triangle pressure and shear of a finished query run with want_panels:
 * pressure_i = -F_i . n_i / A_i, shear_i = |F_i - (F_i . n_i) n_i| / A_i
 * (Pa; n_i the geometric unit normal, F_i the force on triangle i).  Host
 * buffers of n_tri doubles (either may be NULL).  Releases the query's panel
 * memory.  Errors: ENOTFOUND, EINVAL (n_tri mismatch). */
tpmc_status tpmc_panels(tpmc_ctx* ctx, tpmc_query_id query, double* pressure, double* shear, uint32_t n_tri);

/* The per-triangle momentum sums behind tpmc_panels (§II.A: the force is the
 * weighted sum of the momentum the particles deliver): dv_q, a host buffer of
 * [n_tri][3] int64, receives for each triangle the sum over its hits of
 * (v_in - v_out) in units of tpmc_result.fixed_quantum (c_mp units), the same
 * integers whose sum over triangles is tpmc_result.sum_dv_q, bit for bit.  The
 * force on triangle i in N is dv_q[i] * fixed_quantum * weight * m * c_mp.
 * Keeps the panel memory, so tpmc_panels may follow.
 * Errors: ENOTFOUND (no panel loads kept for the query), EINVAL (NULL dv_q,
 * n_tri mismatch), ECUDA. */
tpmc_status tpmc_panel_sums(tpmc_ctx* ctx, tpmc_query_id query, int64_t* dv_q, uint32_t n_tri);

/* Same as tpmc_trace and also fills per-particle records (verification).
 * Errors as tpmc_trace, plus EINVAL for K > 64 or N > 2^26. */
tpmc_status tpmc_trace_records(tpmc_ctx* ctx, tpmc_mesh_id mesh, const tpmc_params* params, uint64_t N,
                               tpmc_records* records, tpmc_result* out);

/* Batched sweep: K queries that differ from `base` only in flow direction and
 * speed ratio, in one persistent launch.  h_dirs: host [K][3]; h_S: host [K]
 * speed ratios (V = S c_mp); either may be NULL, and then every item takes
 * base's direction or speed.  Item k uses stream_id = base->stream_id + k.
 * Per-panel loads are not kept.  Results in h_out[K].
 * Errors as tpmc_trace; EINVAL for K = 0 or K > 2^24. */
tpmc_status tpmc_sweep(tpmc_ctx* ctx, tpmc_mesh_id mesh, const tpmc_params* base, const double* h_dirs,
                       const double* h_S, uint32_t K, uint64_t N_each, tpmc_result* h_out);

/* Device-resident form of tpmc_sweep: d_dirs, d_S and d_out are device
 * buffers; the call only enqueues work on the context's stream and returns.
 * Per-item input errors are reported in d_out[k].status. */
tpmc_status tpmc_sweep_device(tpmc_ctx* ctx, tpmc_mesh_id mesh, const tpmc_params* base, const double* d_dirs,
                              const double* d_S, uint32_t K, uint64_t N_each, tpmc_result* d_out);

/* Batched sweep that allocates no memory (the paper has no counterpart: this
 * serves callers that may not allocate device memory after start-up, such as
 * real-time control loops, code whose device memory belongs to a framework's
 * own pool, or code that must keep a fixed footprint).  Same inputs and
 * results as tpmc_sweep with host buffers (h_dirs [K][3], h_S [K] or NULL,
 * h_out [K]) and the same behaviour: an item rejected by its set-up reports
 * that in h_out[k].status, and h_out[k].ms is the call's wall time; per-panel
 * loads are not kept.  Its scratch is one fixed device
 * array of the library (64 queries, about 170 KB), held by every GPU that
 * loads the library until the process exits.  The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress, which also
 * loads the library's device code there), so make that first call before any
 * stream capture.  All calls on a device share the array; each call clears
 * what must start at zero, and calls that overlap on the GPU race on it.
 * Errors: EINVAL for K = 0 or K > 64, otherwise as tpmc_sweep. */
tpmc_status tpmc_sweep_noalloc(tpmc_ctx* ctx, tpmc_mesh_id mesh, const tpmc_params* base, const double* h_dirs,
                               const double* h_S, uint32_t K, uint64_t N_each, tpmc_result* h_out);

/* ---- serving: continuous batching over resident meshes -------------------- */

/* Queues a query; a scheduler thread admits it when a slot and memory are
 * free and traces it in launches shared with the other queries in flight.
 * Errors: EINVAL/ENOTFOUND as tpmc_trace, EBUSY when the queue is full. */
tpmc_status tpmc_submit(tpmc_ctx* ctx, tpmc_mesh_id mesh, const tpmc_params* params, uint64_t N,
                        tpmc_query_id* out);

/* Waits up to timeout_ms (0: do not wait; < 0: forever) for a submitted query
 * and returns its result (out->ms is the latency from submit to completion).
 * Errors: ETIMEOUT (not finished; poll again), ENOTFOUND. */
tpmc_status tpmc_poll(tpmc_ctx* ctx, tpmc_query_id query, int timeout_ms, tpmc_result* out);

/* ---- schedule ------------------------------------------------------------ */

/* Chooses the trace kernel's BVH layout and launch schedule for `mesh` (the
 * paper's closest-hit ray tracing, §II.A, on this GPU), in three stages:
 *   1. BVH width 2, 4 or 8 (the mesh is laid out again from the context's
 *      copy; the fastest layout replaces the mesh's own unless queries in
 *      flight use it, and later loads of meshes of its size class use it);
 *   2. threads per block, resident blocks per SM, the traversal-round refill
 *      threshold and the BVH nodes staged in shared memory (binary trees);
 *   3. particles per lane: a fixed number of ids a warp takes per fetch.
 * Each candidate runs a trial sweep of `params` over eight flow directions
 * (params->dir, the six axes and a diagonal) of N_trial / 4 and then N_trial
 * particles in all, scored by the marginal rate between the two so that
 * fixed per-launch costs do not decide (N_trial of a few million or more keeps
 * the difference above the noise); a candidate must beat the untuned schedule
 * by 1 %.  The schedule is kept for meshes of the size class and this kernel
 * variant.  `best` (may be NULL) receives it.
 * Errors: as tpmc_trace; EINVAL for N_trial = 0 or > 2^30; ENOMEM when a
 * layout does not fit the memory budget (that width is then skipped). */
tpmc_status tpmc_tune(tpmc_ctx* ctx, tpmc_mesh_id mesh, const tpmc_params* params, uint64_t N_trial,
                      tpmc_launch* best);
tpmc_status tpmc_set_launch(tpmc_ctx* ctx, const tpmc_launch* cfg);
tpmc_status tpmc_get_launch(tpmc_ctx* ctx, tpmc_mesh_id mesh, uint32_t precision, tpmc_launch* out);

/* ---- measurement ---------------------------------------------------------- */

/* Measures on the context's device the two ceilings of the trace kernel's
 * roofline (the kernel works in FP32 on node and triangle data that stays in
 * L1/L2):
 *   *fp32_tflops  FP32 FMA rate of independent dependent-FMA chains on every
 *                 SM, 2 flops per FMA, best of 5 launches;
 *   *l2_read_gbs  read bandwidth of a 32 MiB buffer streamed 64 times from L2
 *                 with loads that bypass L1, best of 5 launches.
 * Runs on the context's stream and waits for it; takes about 50 ms; holds
 * 33 MiB of the context's memory budget during the call.
 * Errors: EINVAL (NULL argument), ENOMEM (budget), ECUDA. */
tpmc_status tpmc_measure_ceilings(tpmc_ctx* ctx, double* fp32_tflops, double* l2_read_gbs);

#ifdef __cplusplus
}
#endif
#endif /* TPMC_H */
