/*
 * pdcloth -- GB300 (sm_103a) projective-dynamics cloth stepper, C ABI.
 *
 * Implements the per-time-step solve of Lan et al., "Efficient GPU Cloth
 * Simulation with Non-distance Barriers and Subspace Reuse" (arXiv
 * 2403.19272): the implicit-Euler variational problem of Sec. 3
 * (Eq. var_barrier) solved by local-global (LG) iterations (Eq. local /
 * Eq. global), with
 *   - non-distance barrier (NDB) collision weights w = k*K^a, Eq. (exp);
 *   - partial CCD (Sec. 4.1, Eq. collision_judge / Eq. query) to update the
 *     weights every LG iteration, exact CCD and the alpha*t_TOI line search
 *     filter for the penetration-free guarantee (Alg. 1, Sec. 7);
 *   - the subspace-reuse correction of Sec. 5 (Eq. subspace_global,
 *     Eq. subspace_collision, Eq. uu) followed by Jacobi relaxation of the
 *     high-frequency residual (Eq. high_frequency_residual);
 *   - the two-subspace scheme of Sec. 7 (a basis of r_warm modes used
 *     without collision springs, its first r_reuse columns with them).
 *
 * Conventions for every entry point
 *   - Every call returns a pdc_status; details of the last failure are
 *     returned by pdc_last_error(handle) (a static string for a NULL
 *     handle).  No call aborts the process.
 *   - The library owns all device memory it allocates (cudaMalloc on the
 *     current device at pdc_create).  The caller owns every buffer it
 *     passes in and out; arguments named on_device select whether a pointer
 *     is a device pointer (1) or a host pointer (0).  Host buffers are only
 *     read or written during the call.
 *   - Positions and velocities are float32, row-major [count][3] (x, y, z
 *     interleaved).  Index arrays are int32.
 *   - Collision vertex ids: cloth vertices 0..nv-1 first, then each
 *     obstacle's vertices in the order obstacles were added.  Collision
 *     triangle ids likewise (cloth triangles first).
 *   - pdc_step is ordered on the stream given to pdc_create (NULL = legacy
 *     default stream) and returns after the step has finished on the GPU.
 *   - Not thread safe per handle; different handles are independent.
 */
#ifndef PDCLOTH_H
#define PDCLOTH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pdc_ctx *pdc_handle;

typedef enum {
    PDC_OK = 0,
    PDC_ERR_ARG = 1,        /* invalid argument (NULL, size, range, dt mismatch) */
    PDC_ERR_CUDA = 2,       /* a CUDA runtime call failed                        */
    PDC_ERR_NUMERIC = 3,    /* NaN/Inf or a failed factorisation; state rolled back */
    PDC_ERR_TIMEOUT = 4,    /* a bounded device wait ran out                      */
    PDC_ERR_DEGENERATE = 5, /* zero-area rest triangle or bad topology           */
    PDC_ERR_STATE = 6,      /* call out of order (e.g. no mesh)                  */
    PDC_ERR_CAPACITY = 7    /* a candidate / hash buffer could not be grown      */
} pdc_status;

/* Mesh given to pdc_create (copied; host pointers). */
typedef struct {
    const float *verts;   /* [nv][3] rest (= initial) positions              */
    int32_t nv;
    const int32_t *tris;  /* [nt][3] vertex ids, consistently oriented        */
    int32_t nt;
    const int32_t *pins;  /* [npins] vertex ids held by Dirichlet conditions  */
    int32_t npins;
} pdc_mesh_desc;

/* Material (Tab. 1 columns rho_m and kappa).  Stretch energy per triangle
 * k_stretch*A_t/2 |F - R|^2 with R the closest 3x2 matrix with orthonormal
 * columns; bending per interior edge (3 k_bend/(A_1+A_2))/2 |sum_j K_j x_j -
 * s_hat|^2 with cotangent weights K and s_hat keeping the rest magnitude. */
typedef struct {
    double density;   /* kg / m^2 */
    double k_stretch;
    double k_bend;
} pdc_material;

/* Solver settings.  Fill with pdc_default_params() and override. */
typedef struct {
    double dt;               /* time step h (s); the basis depends on it         */
    double gravity[3];       /* f_ext = m g                                      */
    double k_ndb_scale;      /* k of Eq. (exp) = k_ndb_scale * mean(diag H)      */
    double K_ndb;            /* growth base K of Eq. (exp) (paper: 2)            */
    int32_t a_max;           /* cap on the life-span counter a                   */
    double alpha_ls;         /* line-search factor alpha (paper: 0.8)            */
    double d_hat;            /* gap of the activity test and contact target (m); <= 0: automatic */
    double eta_ccd;          /* exact-CCD contact distance (m)                   */
    double tol_outer;        /* ||dx||_inf / bbox-diagonal between outer passes  */
    double tol_inner;        /* ||dx||_inf / bbox-diagonal between inner iterations */
    double tol_rel_residual; /* > 0: inner loop stops when the PD residual falls
                                below this fraction of the residual at z        */
    int32_t max_outer, max_inner, warm_iters;
    int32_t jacobi_sweeps;   /* Jacobi sweeps per solve cycle                    */
    double jacobi_omega;     /* Jacobi damping; <= 0: automatic                  */
    int32_t solve_cycles;    /* subspace correction + sweeps per LG iteration    */
    int32_t r_warm;          /* basis size used without collision springs (0: none) */
    int32_t r_reuse;         /* leading columns used with collision springs
                                (<= 512; above 128 the reduced system is
                                factored by blocks over many CTAs)           */
    int32_t precision;       /* 0: plain FP32; 1: mixed with a BF16 basis; 2:
                                mixed with an FP16 basis scaled by a power of two
                                (its rounding noise carries ~2^-6 of the BF16
                                noise's H-energy).  Mixed forms: 16-bit basis on
                                the tensor cores, FP64 reduced solves            */
    int32_t samples_vt;      /* partial-CCD sample pattern: 0, 1 or 3            */
    int32_t samples_ee;      /* partial-CCD sample pattern: 0, 1 or 4            */
    int32_t collisions;      /* 0: no collision handling at all                  */
    int32_t fixed_iters;     /* 1: run exactly warm/max_outer/max_inner iterations */
    int32_t eig_iters;       /* filtered subspace iterations building the basis  */
    uint64_t seed;           /* seed of the basis start block                    */
    int32_t accel;           /* acceleration of the LG iterates (ignored when
                                fixed_iters = 1): 0 none; 1 Chebyshev
                                semi-iteration; 2 Anderson mixing of depth
                                aa_depth                                          */
    double accel_rho;        /* spectral radius for accel; <= 0: estimated from the
                                residual decay of the first iterations of a pass */
    int32_t sweep_kind;      /* 0: damped Jacobi sweeps; 1: Jacobi-preconditioned
                                Chebyshev iteration of jacobi_sweeps steps over the
                                spectrum interval [b / cheb_ratio, b] of D^-1 A   */
    double cheb_ratio;       /* interval ratio for sweep_kind 1 (> 1)            */
    int32_t aa_depth;        /* history length for accel = 2 (1..8)              */
    int32_t tensor_cores;    /* mixed form: 1 runs the full-basis projection and
                                lift on the tcgen05 tensor cores (BF16 basis, FP32
                                operand split into two BF16 parts, FP32
                                accumulation); 0 uses the CUDA-core kernels      */
    double bp_reuse;         /* > 0: the first broad phase of a step runs with the
                                gap d_hat + 2 mu, mu = bp_reuse * d_hat, and later
                                full CCDs of the step filter its candidate list
                                (same pairs, same order as a fresh pass) while
                                every vertex stays within 0.9 mu of its swept box;
                                0 (default): a hash pass for every full CCD     */
    int32_t launch_overlap;  /* 1 (default): the kernels of an LG iteration (element
                                forces and residual, tensor-core projection,
                                reduction and lift, Chebyshev steps, Anderson
                                mixing) are launched as programmatic dependents
                                of the kernel before them, so each launch and
                                its block scheduling overlap the previous
                                kernel's tail (a kernel waits for its
                                predecessor's results before touching them); 0:
                                plain stream order.  Results are identical.    */
    double rf_toi;           /* residual forwarding (Sec. 6, end of Alg. 1): when
                                the exit time of impact is below rf_toi, up to
                                rf_iters more LG iterations of the step's problem
                                run from the filtered positions with every active
                                constraint at weight k (a = 0) and no CCD; the
                                change dx shifts the next step's z by 2 dx
                                (Eq. z_rf).  0 (default): off                   */
    int32_t rf_iters;        /* cap on those iterations (exact count when
                                fixed_iters = 1); they stop once the largest
                                change is below tol_inner * bbox diagonal       */
    int32_t loop_control;    /* who takes the stopping tests of the LG loops
                                (warm start, inner loops): the relative
                                residual, stagnation, step-change and cap tests.
                                1 (default): a one-thread kernel on the device
                                after each residual, the loop run as one CUDA
                                graph whose conditional while node repeats the
                                iteration (graph_unroll per pass); the fastest
                                of the four on the 512 x 512 sheet.  2: the
                                same device tests; the host enqueues the
                                iterations ahead (loop_ahead) and reads the
                                decisions from host-mapped memory, with no
                                stream synchronisation per iteration; kernels
                                enqueued past the loop's end return at once.
                                3: as 2, each iteration launched as one CUDA
                                graph (captured once per loop kind).  0: the
                                host reads each iteration's residual back and
                                decides (also while profiling, with PDC_LOG or
                                PDC_SYNC_CHECK, or with accel = 1).  Same
                                kernels in the same order in every mode.        */
    int32_t pccd_adaptive;   /* 1: the partial CCD tests, instead of the fixed
                                samples_vt / samples_ee patterns, the t = 0
                                closest point and a lattice of spacing 1/m over
                                the pair's parameters, m = ceil(1 / (sqrt(2)
                                rho*)) from the bound rho* of Eq. (sample_bound)
                                (Sec. 4.1; with alpha_ls as alpha): every pair
                                colliding before alpha of the step is flagged
                                unless m was capped.  0 (default): fixed
                                patterns                                          */
    int32_t pccd_max_axis;   /* cap on m (1..256, default 64)                    */
    int32_t instance_line_search; /* batched form: 1 gives every instance its own
                                step fraction s_k = alpha * t_k (1 without an
                                impact), t_k the smallest time of impact of the
                                pairs with a vertex in instance k (a pair that
                                spans two instances counts for both); its
                                attached obstacles (pdc_set_obstacle_instance)
                                move with it.  Needs every obstacle attached,
                                else the union's single fraction is used.  0
                                (default): one fraction for the union          */
    int32_t autotune;        /* 1: the first step picks the launch shapes of the
                                hot kernels by timing every candidate on the
                                handle's own data (CUDA events; see
                                pdc_tuning), the broad phase its grid and
                                block shape on its 8th pass (the first steps
                                see the cloth nearly at rest); results do not
                                depend on the choice beyond the order of float
                                atomics.  0 (default): fixed shapes            */
    int32_t graph_unroll;    /* loop_control = 1: LG iterations per pass of the
                                while node (1..8, default 1): each pass
                                relaunches its body on the device, at a cost
                                that grows with the body's node count; the
                                kernels of iterations after the loop's end
                                return at once                                   */
    int32_t loop_ahead;      /* loop_control = 2, 3: LG iterations the host
                                enqueues beyond the last one whose decision it
                                has read (0..2, default 1).  Each one the loop
                                ends before costs a pass of kernels that return
                                at once; 0 leaves the device waiting for the
                                host between iterations                         */
    int32_t cheb_source;     /* matrix the Chebyshev steps read: -1 (default)
                                the patch tiles when they exist, else the row
                                tiles (autotune: the fastest of those built);
                                0 the ELL arrays; 1 the row tiles; 2 the patch
                                tiles; 3 two steps a launch over patches
                                widened by a second ring (a source that is not
                                built falls back to the next simpler one).
                                Same arithmetic in the same order in every
                                source                                          */
    int32_t residual_patch;  /* 1 (default): the element projections and the
                                residual of an LG iteration in one kernel per
                                mesh patch (each patch's element forces in
                                shared memory); 0: two kernels through
                                per-corner force arrays in device memory.
                                Same terms summed in the same order             */
} pdc_params;

/* Per-step statistics (Tab. 1 columns: LG iterations, #Col., B|N|P|F). */
typedef struct {
    int32_t warm_iters, outer_iters, inner_iters;
    int32_t contact_iters;       /* LG iterations that ran the collision-spring
                                    path of the global solve (when the residual
                                    is read back: only those with at least one
                                    contact vertex)                              */
    int64_t n_candidates;        /* broad-phase pairs of the last full CCD       */
    int64_t n_active;            /* active NDB constraints after the step        */
    int64_t n_contact_vertices;  /* vertices with a collision spring (last iter) */
    double t_toi;                /* exit time of impact (2 = none)               */
    double s_line_search;        /* applied step fraction (1 or alpha*t_TOI)     */
    double rho0;                 /* PD residual at z                              */
    double rel_residual;         /* last measured residual / rho0                 */
    double ms_step, ms_broad, ms_narrow, ms_lg; /* host wall time per phase (ms) */
    int32_t overflow_retries;    /* buffer regrowths during this step            */
    int32_t bp_reused;           /* full CCDs whose candidates were filtered from
                                    the step's first broad phase (bp_reuse)      */
    int32_t rf_iters;            /* residual-forwarding LG iterations run at the
                                    end of this step (0: not triggered)          */
    int32_t device_loops;        /* LG loops of this step whose stopping tests
                                    ran on the device (loop_control 1, 2 or 3) */
} pdc_stats;

/* Launch shapes in use and, after an autotuned first step, the measured
 * time (ms) of every candidate. */
typedef struct {
    int32_t tuned;           /* 1 once the first step has tuned (autotune = 1)   */
    int32_t residual_block;  /* threads per block of the element-force and
                                residual kernels (candidates 64, 128, 256)      */
    int32_t cheb_tile;       /* Chebyshev steps read 2 (default when built): the
                                matrix tiles of compact patches of the rest
                                mesh, delta staged with the patch's halo in
                                shared memory; 3: two steps a launch over
                                patches widened by a second ring; 1: the
                                TMA-staged tiles of consecutive rows; 0: the
                                ELL arrays (candidates 1, 0, 2, 3)              */
    int32_t pair_blocks;     /* blocks of the per-pair kernels (152 x 2, 4, 8, 16) */
    int32_t cell_warps;      /* warps per block of the broad phase's cell-pair
                                kernel (candidates 4, 8, 16)                     */
    float residual_ms[3];
    float cheb_ms[4];
    float pair_ms[4];
    float cell_ms[3];
    float cell_grid;         /* factor of the broad phase's cell side over the
                                mean triangle extent (candidates 1, 1.5, 2);
                                the pair lists do not depend on it             */
    float grid_ms[3];
} pdc_tuning;

/* Defaults: dt 1/200, g = (0,0,-9.8), K = 2, a_max 20, alpha 0.8, automatic
 * d_hat, eta 1e-9, tolerances 1e-3 / 5e-2, 4 outer x 32 inner, 5 warm
 * iterations, 4 damped Jacobi sweeps (automatic omega), 1 cycle, no basis,
 * FP32, samples 3/4, collisions on, no LG acceleration, tensor cores for the
 * mixed forms, dependent launches on, broad-phase reuse and residual
 * forwarding off, LG-loop tests on the device (loop_control 1). */
void pdc_default_params(pdc_params *p);

/* Build the solver for one cloth mesh (Sec. 3; Eq. (global) rest matrix,
 * lumped masses, rest operators; Sec. 7 basis precomputation of the r_warm
 * lowest eigenvectors of the rest matrix).  Fails with PDC_ERR_DEGENERATE on
 * zero-area triangles or edges shared by more than two triangles.
 * stream: a cudaStream_t or NULL. */
pdc_status pdc_create(const pdc_mesh_desc *mesh, const pdc_material *mat, const pdc_params *params,
                      void *stream, pdc_handle *out);

/* Batched form: `count` independent cloths (meshes[k] with materials[k];
 * host arrays, copied) advanced together as one system, so that every kernel
 * of a step is one launch over all instances, whatever their sizes.  The
 * union's vertices are numbered instance after instance (instance k starts
 * at the sum of the vertex counts of instances 0..k-1); positions, pins,
 * states and obstacles use that numbering, and every other call applies to
 * the union unchanged.  Readings of the batched form: the iteration stops
 * when the union meets the convergence test, the line search takes one step
 * fraction for all instances (an impact in one shortens every instance's
 * step), and the basis is built for the union's block-diagonal matrix.
 * Place instances apart: a collision pair spanning two instances is handled
 * like any other.  Errors as pdc_create. */
pdc_status pdc_create_batch(int32_t count, const pdc_mesh_desc *meshes, const pdc_material *materials,
                            const pdc_params *params, void *stream, pdc_handle *out);

/* Add a kinematic (infinite-mass) triangle obstacle; host arrays copied.
 * Must be called before the first pdc_step.  Its current and target
 * positions start at verts. */
pdc_status pdc_add_obstacle(pdc_handle h, const float *verts, int32_t nv, const int32_t *tris, int32_t nt,
                            int32_t *out_id);

/* Batched form: attach obstacle id to instance (0..count-1; -1 detaches):
 * with instance_line_search its motion within a step is scaled by that
 * instance's step fraction, so that every pair between the instance's cloth
 * and the obstacle stays on the linear motion its CCD checked.
 * PDC_ERR_ARG for a bad id or instance or a handle that is not batched. */
pdc_status pdc_set_obstacle_instance(pdc_handle h, int32_t id, int32_t instance);

/* Target position of obstacle id at the end of the next step: m4x4 (row
 * major, host) applied to the obstacle's verts as given at pdc_add_obstacle.
 * Within a step the obstacle moves linearly from its current position. */
pdc_status pdc_set_obstacle_transform(pdc_handle h, int32_t id, const float *m4x4);

/* Pinned positions [npins][3] at the end of the next step (Dirichlet). */
pdc_status pdc_set_pin_targets(pdc_handle h, const float *xyz, int32_t on_device);

/* Overwrite / read the state x*, v* ([nv][3] each; v may be NULL on set to
 * zero it).  The current positions must be free of intersections (Sec. 3:
 * the barrier method starts from a feasible state).  Setting the state
 * discards a pending residual-forwarding displacement (rf_toi). */
pdc_status pdc_set_state(pdc_handle h, const float *x, const float *v, int32_t on_device);
pdc_status pdc_get_state(pdc_handle h, float *x, float *v, int32_t on_device);

/* Replace the library's basis by a caller-supplied one: U host [nv][r]
 * float32 row-major (rows of pinned vertices are ignored and taken as 0),
 * r >= r_reuse.  The reduced matrices U^T H U are recomputed from it
 * (Eq. subspace_global with the basis actually used). */
pdc_status pdc_set_basis(pdc_handle h, const float *U, int32_t r);

/* Copy the basis in use (float32 [nv][r_warm]) and its reduced matrix
 * U^T H U (float64 [r_warm][r_warm]) to host buffers (either may be NULL). */
pdc_status pdc_get_basis(pdc_handle h, float *U, double *A0);

/* Advance one time step (Alg. 1).  dt must equal params.dt (PDC_ERR_ARG
 * otherwise: H and the basis depend on h).  On PDC_ERR_NUMERIC the state is
 * left at x*, v*. */
pdc_status pdc_step(pdc_handle h, double dt);

/* Current cloth positions [nv][3]. */
pdc_status pdc_get_positions(pdc_handle h, float *out, int32_t on_device);

/* Displacement u [nv][3] of the last step: inside a step the iterate is
 * carried as x = x* + u (x* the state the step started from), and the step
 * ends at x_new = x* + u, stored as the float32 positions fl32(x* + u).
 * With x* (the positions before the step) and u both float32, x* + u is the
 * step's final iterate exactly (in FP64), free of the rounding of the
 * stored positions, which for a stiff cloth can exceed the residual
 * tolerance.  Zero before the first step and after pdc_set_state. */
pdc_status pdc_get_displacement(pdc_handle h, float *u, int32_t on_device);

/* Statistics of the last step. */
pdc_status pdc_get_stats(pdc_handle h, pdc_stats *out);

/* Candidate pairs of the last full CCD of the last step with their
 * non-distance-barrier states (Sec. 4, Eq. exp): prim [cap][2] the pair's
 * primitives (VT: collision vertex, collision triangle; EE: two edge ids,
 * first < second, edges numbered in ascending (min vertex, max vertex)
 * order), kinds [cap] (0 VT, 1 EE), state [cap] (bit 7: active; bits 0-6:
 * the life-span counter a, the weight being k K^a).  VT pairs come first,
 * each kind sorted by its primitive ids.  *count receives the number of
 * pairs; only the first cap are written.  0 pairs before the first step or
 * without collision handling.  Host buffers. */
pdc_status pdc_get_pairs(pdc_handle h, int32_t *prim, int32_t *kinds, uint8_t *state, int64_t cap, int64_t *count);

/* Launch shapes (autotune) of the handle. */
pdc_status pdc_get_tuning(pdc_handle h, pdc_tuning *out);

/* Copy bandwidth (GB/s, read plus written bytes) of a working set of
 * `bytes`, half of it read and half written per pass, measured by one
 * persistent kernel that makes `passes` passes over it on `stream` (a
 * cudaStream_t or NULL), timed with CUDA events, after two untimed passes.
 * A working set well below the L2 size (129 MB on GB300) gives the L2 copy
 * bandwidth that bounds the kernels whose data stays in L2.  The paper has
 * no counterpart: this supplies the roofline of those kernels.  Allocates
 * and frees its buffers (on the current device); needs no handle (errors:
 * pdc_last_error(NULL)).  PDC_ERR_ARG unless 1 KiB <= bytes <= 64 GiB and
 * passes >= 1. */
pdc_status pdc_measure_copy_bandwidth(int64_t bytes, int32_t passes, void *stream, double *gbs);

/* Free everything owned by the handle (NULL is ignored). */
void pdc_destroy(pdc_handle h);

/* Last error message of the handle, or of the last failed pdc_create when
 * h is NULL.  Never NULL. */
const char *pdc_last_error(pdc_handle h);

/* Per-kernel device time of the launches made while profiling is on: a
 * CUDA event pair on the library's stream around every launch (around each
 * run of back-to-back Chebyshev steps of one global solve, which counts as
 * that many launches), resolved at the end of each pdc_step.  algo_bytes is
 * the algorithmic traffic of those launches (the minimum bytes the method
 * must move for them: element data, vertex streams, sparse-matrix entries,
 * basis rows; gathered neighbour re-reads not counted).  Profiling adds a
 * few microseconds per event pair. */
typedef struct {
    char name[32];
    int64_t launches;
    double total_ms;
    double algo_bytes;
} pdc_kernel_time;

/* Diagnostics read from the environment at pdc_create: PDC_LOG (any value)
 * prints per-iteration residuals, pass decisions and retries to stderr;
 * PDC_SYNC_CHECK (any value) synchronises the stream after every profiled
 * region and fails the call with PDC_ERR_CUDA naming the region if a CUDA
 * error is pending (slow; for locating a fault); PDC_BP_CAPACITY (a positive
 * integer) sets the initial capacity of the broad-phase candidate lists, in
 * pairs of each kind, instead of the size-based default (small values make
 * the first steps regrow the lists, for testing that path). */

/* enable = 1 starts profiling and clears the accumulated times; 0 stops. */
pdc_status pdc_set_profiling(pdc_handle h, int32_t enable);
/* Copies at most cap entries; *count receives the number of kernel kinds. */
pdc_status pdc_get_kernel_times(pdc_handle h, pdc_kernel_time *out, int32_t cap, int32_t *count);

/* --------------------------------------------------------------------------
 * Stage entry points.  Each runs exactly the kernels pdc_step uses for one
 * stage, on caller data, so that every stage can be checked on its own.
 * Collision positions cover all collision vertices (cloth, then obstacles).
 * ------------------------------------------------------------------------ */

/* Broad phase (the candidate set of the CCD of Sec. 4 / Alg. 1): all
 * vertex-triangle pairs (v, t), v not in t, and edge-edge pairs sharing no
 * vertex, not both kinematic, whose swept boxes over x0 -> x1 meet under
 * lo_a <= fl32(hi_b + d_hat) and lo_b <= fl32(hi_a + d_hat) per axis.
 * Output: vt [cap_vt][2] (v, t) sorted by (v, t); ee [cap_ee][4] vertex ids
 * (a, b, c, d), a < b, c < d, sorted by edge ids.  Counts are returned even
 * when they exceed the caps (then only cap entries are written).
 * x0, x1: host [nvc][3], nvc = cloth + obstacle vertices. */
pdc_status pdc_op_broadphase(pdc_handle h, const float *x0, const float *x1, int32_t *vt, int64_t cap_vt,
                             int64_t *n_vt, int32_t *ee, int64_t cap_ee, int64_t *n_ee);

/* Exact CCD (Sec. 4, Eq. intersect; Alg. 1 FullCCD) per pair: first t in
 * [0,1] at which the primitives touch (distance <= eta_ccd at a root or
 * critical point of the coplanarity cubic), 2 if none.  quads [np][4]
 * vertex ids (VT: v,a,b,c; EE: a,b,c,d), kinds [np] 0 = VT, 1 = EE.  Host. */
pdc_status pdc_op_ccd(pdc_handle h, const float *x0, const float *x1, const int32_t *quads,
                      const int32_t *kinds, int64_t np, double *toi);

/* Partial CCD (Sec. 4.1): active[i] = 1 when Q(lambda_s) <= d_hat*|p2^0 -
 * p1^0| at some sample (the t=0 closest point plus the samples_vt /
 * samples_ee pattern).  Host arrays as in pdc_op_ccd. */
pdc_status pdc_op_partial_ccd(pdc_handle h, const float *x0, const float *x1, const int32_t *quads,
                              const int32_t *kinds, int64_t np, int32_t *active);

/* Collision springs (Sec. 5.1, A_i = B_i = Id) of the given active pairs
 * with weights w [np]: per cloth vertex the weight sum cw [nv] and the
 * force sum cf [nv][3] = sum_i w_i (y_ij - x_j), targets from the t=0
 * closest points on x0 and the constraint (p2 - p1).n0 >= d_hat at x. */
pdc_status pdc_op_contact(pdc_handle h, const float *x0, const float *x, const int32_t *quads,
                          const int32_t *kinds, const float *w, int64_t np, float *cw, float *cf);

/* PD residual r = b(x) - (H + diag(cw)) x of Eq. (global) with the local
 * projections at x, over cloth vertices (0 on pinned rows); cw, cf as
 * returned by pdc_op_contact (NULL = no contact).  Host arrays. */
pdc_status pdc_op_residual(pdc_handle h, const float *x, const float *z, const float *cw, const float *cf,
                           float *r);

/* One global solve as run inside an LG iteration: residual at x, then
 * `cycles` times {subspace correction in span(U[:, :r]) with the reduced
 * matrix U^T (H + diag(cw)) U (Eq. subspace_collision / uu), `sweeps`
 * Jacobi sweeps (Eq. high_frequency_residual)}; writes x_out = x + delta.
 * r = 0 skips the correction; 0 <= r <= min(r_warm, 512).  Host arrays. */
pdc_status pdc_op_global_solve(pdc_handle h, const float *x, const float *z, const float *cw, const float *cf,
                               int32_t r, int32_t cycles, int32_t sweeps, float *x_out);

/* Subspace projection g = U[:, :r]^T v (the U^T r of Eq. subspace_global)
 * with the handle's basis, as run in the LG iterations without collision
 * springs: on the tcgen05 tensor cores when params.precision = 1,
 * params.tensor_cores = 1 and the basis row stride is a multiple of 128
 * (<= 256), else on the CUDA cores.  v: host [nv][3] float32 (pinned rows
 * ignored through U's zero rows); g: host [r][3] float64; 0 < r <= r_warm. */
pdc_status pdc_op_project(pdc_handle h, const float *v, int32_t r, double *g);

/* Lift out = U[:, :r] q (the U q of Eq. subspace_collision), same path
 * selection as pdc_op_project.  q: host [r][3] float64 (used as float32);
 * out: host [nv][3] float32. */
pdc_status pdc_op_lift(pdc_handle h, const double *q, int32_t r, float *out);

/* Size of the one statically allocated device array (per device) that
 * pdc_op_contact_noalloc uses for its temporaries. */
#define PDC_NOALLOC_SCRATCH_BYTES (8u << 20)

/* Allocation-free variant of pdc_op_contact.  The paper has no counterpart:
 * this is a library-integration entry point, not part of the method.
 *
 * It computes exactly what pdc_op_contact computes for the given pairs and
 * weights, but allocates no device memory: no cudaMalloc / cudaFree and no allocating
 * library routine.  It is meant for callers that cannot let a library
 * allocate inside a call -- a process whose caching allocator already holds
 * nearly all free device memory (a cudaMalloc there fails, or forces the
 * allocator to give memory back), or a latency-bound loop, since cudaFree
 * synchronises the whole device and stalls every other stream.
 *
 * All pointers are DEVICE pointers on the current device:
 *   x0, x   [nv_all][3] float32 collision-vertex positions (cloth, then
 *           obstacles), t = 0 of the pairs and the evaluation positions;
 *   quads   [np][4] int32 vertex ids, 16-byte aligned; kinds [np] int32
 *           (0 = VT, 1 = EE); w [np] float32 weights;
 *   cw      [nv] float32 out: per cloth vertex the weight sum (nv = cloth
 *           vertices);
 *   cf      [nv][3] float32 out: per cloth vertex sum_i w_i (y_ij - x_j).
 * stream: a cudaStream_t on the current device (NULL = the handle's stream).
 *
 * Scratch: the temporaries (float4 copies of x0 and x, the force
 * accumulator, the active-pair list and two counters) live in one file-scope
 * device array of PDC_NOALLOC_SCRATCH_BYTES.  They need
 *   32*nv_all + 16*nv + 48*max(np,1) bytes (+ alignment, each part rounded
 *   up to 256 B, + 256 B of counters);
 * larger inputs are rejected with PDC_ERR_CAPACITY before any work is
 * enqueued (use pdc_op_contact for them).  Nothing has to start at zero:
 * the call zeroes its counters, its accumulator and both outputs itself, and
 * cw and cf are overwritten in full.
 *
 * The first call on a device looks the scratch address up with
 * cudaGetSymbolAddress, which can load the library's device code; make that
 * first call before any stream capture on the device.  Every call on one
 * device shares the same scratch, so calls that overlap in time (other
 * threads, other streams, other handles) race and corrupt each other's
 * results: order them on one stream or on the host.
 *
 * Ids and kinds are checked on the device before use (one stream
 * synchronisation): PDC_ERR_ARG if any is out of range.  The remaining work
 * is enqueued on `stream`; cw and cf are valid once it has completed.
 * PDC_ERR_STATE if obstacle topology has not been built. */
pdc_status pdc_op_contact_noalloc(pdc_handle h, const float *x0, const float *x, const int32_t *quads,
                                  const int32_t *kinds, const float *w, int64_t np, float *cw, float *cf,
                                  void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PDCLOTH_H */
