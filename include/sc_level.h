/*
 * sc_level.h -- C ABI of the GB300 stencil / RK4 level library
 * (libsc_level.so).
 *
 * A *level* is a set of non-overlapping boxes on a uniform grid whose points
 * are x0 + n*h with integer n (arXiv 1308.1343, Sec. 2, "Efficient Bounding
 * Box Algebra": bbox / bboxset).  Boxes belong to *domains*; the boxes of a
 * domain tile it exactly.  Each box stores its interior points plus ghost
 * zones of width 2, and the ghost exchange between boxes (periodic images
 * included) is the communication schedule derived from bboxset intersections
 * (Sec. 2, list of operations built on the set algebra).
 *
 * The library evolves the first-order-in-time scalar wave equation
 *     du/dt = pi,   dpi/dt = c2(x) * (L u)
 * with L the 4th-order centred Laplacian
 *     (L u)_i = sum_d ( -u_{i-2e_d} + 16 u_{i-e_d} - 30 u_i + 16 u_{i+e_d}
 *                       - u_{i+2e_d} ) / (12 h^2)
 * (the centred-difference idiom on padded arrays of Sec. 4.3, "Iterators"),
 * by classic fourth-order Runge-Kutta, and differentiates it (adjoint).
 * All arithmetic is FP64 on the GPU; the traversal follows Sec. 3's loop
 * decomposition (tiles, then points within tiles) and its run-time tuning.
 *
 * Conventions for every function:
 *  - Return value: SC_OK (0) or a negative SC_E* code; the matching message
 *    is available from sc_last_error() on the calling thread.  No function
 *    aborts the process, and no kernel traps: device-side problems set a
 *    device error word that the next synchronising call reports as
 *    SC_EDEVICE.  The device state of a level (work lists, coefficients)
 *    is built by its first device call; if that set-up fails, nothing of it
 *    is kept and the next call builds it again.
 *  - Field buffers are caller-owned DEVICE pointers (e.g. torch tensors) of
 *    sc_level_field_size() doubles, 16-byte aligned, in the level layout
 *    below.  The library owns the level object and all of its scratch memory
 *    (stage arrays, checkpoints, work lists, CUDA graphs).
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *    default stream.  Work is enqueued asynchronously unless stated.
 *
 * Level layout (all boxes of all domains in one buffer, box-major):
 *  - Box b with interior extent (nx, ny, nz) is stored as a padded box of
 *    (nx+4) x (ny+4) x (nz+4) points, x fastest, with row pitch
 *    py = roundup(nx+4, 16) doubles and plane pitch pz = py*(ny+4).
 *  - The element index of grid point p of box b is
 *        offset_b + (p.x-lo.x) + (p.y-lo.y)*py + (p.z-lo.z)*pz
 *    for lo-2 <= p < hi+2 on each axis; offset_b (the interior corner lo)
 *    is a multiple of 16, so every interior row starts on a 128-byte line.
 *  - Ghost points are the star-shaped shell: points within 2 of a face
 *    along exactly one axis.  Edge and corner points of the padded box and
 *    row padding are never read or written by the library.
 */
#ifndef SC_LEVEL_H
#define SC_LEVEL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define SC_OK 0
#define SC_EINVAL (-1)   /* bad argument: boxes overlap / do not tile a domain,
                            ghost != 2, misaligned or NULL pointer, bad size */
#define SC_ENOMEM (-2)   /* host or device allocation failed               */
#define SC_ECUDA (-3)    /* a CUDA runtime call failed                      */
#define SC_EDEVICE (-4)  /* a kernel set the device error word (e.g. a
                            non-finite value reached the fixed-point path)  */
#define SC_ENOTSUP (-5)  /* valid request this build does not support        */

/* ---- arithmetic of the Laplacian sum ----------------------------------- */
/* SC_ARITH_FP64:  the 13-term sum is evaluated with FP64 adds and FMAs.
 * SC_ARITH_FIXED: each input is scaled by 2^S (S from the domain-wide
 *   maximum exponent of the field) and truncated to a 64-bit integer; the
 *   integer-weighted sum is then exact and is rounded once to FP64.  The
 *   per-input error is below 2^-54 of the domain's maximum |value|, so
 *   the error in the max norm is about that of the FP64 sum.  Non-finite
 *   inputs set the device error word.  The RK updates are FP64 FMAs in
 *   both modes. */
#define SC_ARITH_FP64 0
#define SC_ARITH_FIXED 1

/* ---- traversal mode of sc_level_rk4_step -------------------------------- */
#define SC_MODE_GRAPH 0    /* one batched launch per kernel over the whole
                              level's work list, a CUDA graph per RK4 step  */
#define SC_MODE_PER_BOX 1  /* one launch per box per kernel, no graph       */
#define SC_MODE_BATCHED 2  /* batched launches without the graph            */
#define SC_MODE_TIMED 3    /* batched launches, each stage and gather kernel
                              bracketed by CUDA events on the stream (see
                              sc_level_kernel_times); for measurement       */

typedef struct sc_box {
    int64_t lo[3], hi[3]; /* half-open [lo, hi) in the level's index space */
    int32_t domain;       /* index into the domain array                    */
    int32_t reserved;     /* must be 0                                      */
} sc_box;

typedef struct sc_domain {
    int64_t lo[3], hi[3]; /* half-open extent of the domain                 */
    double h;             /* grid spacing (same on all axes)                */
    uint32_t periodic;    /* bit d set: periodic along axis d (x=1,y=2,z=4) */
    uint32_t reserved;    /* must be 0                                      */
} sc_domain;

/* One rectangular ghost copy: for every offset o in [0, ext),
 * dst_box(dst_lo + o) = src_box(src_lo + o), coordinates in the level's
 * index space (dst points are ghosts of dst_box, src points interior points
 * of src_box, equal to the ghost points modulo the periodic domain). */
typedef struct sc_copy {
    int32_t src_box, dst_box;
    int64_t src_lo[3], dst_lo[3], ext[3];
} sc_copy;

typedef struct sc_level sc_level;

/* Kernel configuration of one box-size class (chosen by sc_level_autotune or
 * set explicitly).  tile_x, tile_y: points per CTA tile in x and y
 * (tile_x/2 * tile_y == threads per CTA, see sc_level_set_tuning); tile_z:
 * depth of the z-run one work item marches through.  Where a box's extent
 * leaves less than a whole tile, other shapes of the same thread count
 * cover the rest (see sc_level_work_items). */
typedef struct sc_tile {
    int32_t tile_x, tile_y, tile_z, reserved;
} sc_tile;

/* ---- level lifetime ----------------------------------------------------- */

/* Build a level from boxes and domains (host only: validates the level with
 * the bboxset algebra and builds the exchange lists; device state is created
 * on the first call that takes a stream).  ghost must be 2.  Every box must
 * lie in its domain, have edges >= 2, and the boxes of each domain must tile
 * it exactly; one field of the level must hold fewer than 2^31 doubles.  On success *out owns the level (free with sc_level_destroy).
 * Errors: SC_EINVAL (message names the offending box), SC_ENOMEM. */
int sc_level_create(const sc_box* boxes, int32_t nboxes, const sc_domain* doms,
                    int32_t ndoms, int32_t ghost, sc_level** out);

/* Free the level and all library-owned device memory.  Waits for the
 * device to finish work on the level.  NULL is ignored. */
void sc_level_destroy(sc_level* level);

/* ---- layout queries (host only) --------------------------------------- */

/* Number of doubles in one field buffer of this level. */
int sc_level_field_size(const sc_level* level, int64_t* n_doubles);

/* Layout of box `box`: offset = element index of the interior corner lo,
 * dims = interior extent (nx, ny, nz), pitch = (1, py, pz) in doubles. */
int sc_level_box_layout(const sc_level* level, int32_t box, int64_t* offset,
                        int64_t dims[3], int64_t pitch[3]);

int sc_level_num_boxes(const sc_level* level, int32_t* nboxes);

/* Copy the exchange list (all boxes) into out[0..cap); *n receives the total
 * count (call with cap = 0 to size the buffer).  Order: by destination box,
 * then by the order the bboxset sweep emits the rectangles. */
int sc_level_exchange_list(const sc_level* level, sc_copy* out, int64_t cap,
                           int64_t* n);

/* ---- configuration ----------------------------------------------------- */

/* Select the Laplacian arithmetic (SC_ARITH_*) for all later calls. */
int sc_level_set_arith(sc_level* level, int32_t arith);

/* Set the tile of one size class (class index as reported by
 * sc_level_size_classes) and the persistent-grid CTAs per SM (0 = keep).
 * tile_x in {16, 32, 64}, tile_y such that tile_x/2*tile_y == 256,
 * tile_z >= 1.  Invalidates captured graphs. */
int sc_level_set_tuning(sc_level* level, int32_t size_class, const sc_tile* tile,
                        int32_t ctas_per_sm);

/* The tile of one size class as the kernels use it: set by
 * sc_level_set_tuning or sc_level_autotune, else the heuristic default
 * (whose tile_z is final only once the level has device state). */
int sc_level_get_tuning(const sc_level* level, int32_t size_class, sc_tile* tile);

/* RK4 stages per stencil pass of sc_level_rk4_step, sc_level_forward_tape
 * and the forward recomputation of sc_level_backward_tape (default 2).
 * 1: one launch per stage, w_s = y + g_s A w_{s-1} as in the paper's
 *    method-of-lines stage loop.
 * 2: two launches per step.  Only the u-component goes through L and
 *    w_s.u is pointwise in (y.u, w_{s-1}.pi), so by linearity
 *    L w_1.u = L y.u + g_1 L y.pi and L w_3.u = L y.u + g_3 L w_2.pi: pass A
 *    applies L to y.u and y.pi and gives w_2 (and L y.u), pass B applies L to
 *    w_2.u and w_2.pi and gives the new y, every stencil still of radius 2
 *    and every exchange still two points deep (two fields per exchange).
 *    This is loop fusion chosen per run (arXiv 1308.1343, Sec. 3.3, fusing
 *    loops as a tuning option).  Results equal the one-stage form up to
 *    rounding.  sc_box_rk4_step_noalloc always runs one stage per pass.
 * Setting the form fixes it; until then sc_level_autotune tunes both forms
 * and keeps the faster.  Errors: SC_EINVAL for other values. */
int sc_level_set_fusion(sc_level* level, int32_t stages_per_pass);
int sc_level_get_fusion(const sc_level* level, int32_t* stages_per_pass);

/* Staging of the one-stage kernel's raw stencil inputs (the column value
 * two planes ahead and the tile's halo pairs), the GPU form of the paper's
 * compile-time tuning parameters (Sec. 3.3, prefetching as an option):
 *  SC_STAGING_REGISTERS: loaded to registers one plane ahead (46 KB of
 *    shared memory, 4 CTAs per SM);
 *  SC_STAGING_SHARED: copied to shared memory by cp.async with the
 *    pointwise fields (62 KB, 3 CTAs per SM).
 * Results are identical.  The two-stage pass kernels always stage in shared
 * memory (registers are their scarce resource).  Setting it fixes it; until
 * then sc_level_autotune times both for the one-stage form and keeps the
 * faster.  Errors: SC_EINVAL for other values. */
#define SC_STAGING_REGISTERS 0
#define SC_STAGING_SHARED 1
int sc_level_set_staging(sc_level* level, int32_t staging);
int sc_level_get_staging(const sc_level* level, int32_t* staging);

/* Kernels of the two-stage passes (sc_level_set_fusion(2)):
 *  SC_PASS_ONE_ROLE: every warp of a CTA converts, sums and runs the RK
 *    epilogue of its points, one barrier per plane (256 threads, two CTAs
 *    per SM);
 *  SC_PASS_WARP_SPECIALISED: 8 producer warps convert and form the sums,
 *    4 consumer warps run the epilogue, handing each plane's sums over
 *    through a ring of shared-memory slots guarded by mbarriers, so the
 *    FP64 epilogue runs beside the integer work of the next planes (384
 *    threads, two CTAs per SM; the roles take 96 and 48 registers).  Every
 *    wait inside it is bounded (1 s); a wait that gives up ends the kernel
 *    and sets the device error word (SC_EDEVICE at sc_level_sync).
 * Results are bit-identical.  The default is SC_PASS_WARP_SPECIALISED.
 * Setting it fixes it; until then sc_level_autotune tunes the tiles of both
 * and keeps the faster kernel.  Errors: SC_EINVAL. */
#define SC_PASS_ONE_ROLE 0
#define SC_PASS_WARP_SPECIALISED 1
int sc_level_set_pass_kernel(sc_level* level, int32_t kind);
int sc_level_get_pass_kernel(const sc_level* level, int32_t* kind);

/* For tests of failure detection: the next launch of a warp-specialised
 * pass kernel on this level (batched or per-box mode, not a graph captured
 * earlier) withholds the consumers' release of its ring slots, so the
 * producers' bounded wait runs out after 1 s; the kernel returns early and
 * sc_level_sync reports SC_EDEVICE.  The fields it was writing are then
 * undefined.  One shot.  SC_EINVAL unless the level runs the
 * warp-specialised two-stage passes. */
int sc_level_arm_wait_test(sc_level* level);

/* Number of box-size classes and the class of each box (boxes are grouped
 * by interior extent rounded up to a multiple of 8 per axis). */
int sc_level_size_classes(const sc_level* level, int32_t* nclasses,
                          int32_t* class_of_box /* nboxes entries or NULL */);

/* The work items of the level's batched launches, in their launch order:
 * out[6 i .. 6 i + 5] = box, x0, y0, z0 (the item's first point, interior
 * coordinates of its box), number of planes of its z-run, tile_x (the tile
 * is tile_x x 512 / tile_x points), for i < min(cap, n); *n receives the
 * count (cap = 0 sizes the buffer).  Built on the host from the size
 * classes' current tiles (after sc_level_autotune or sc_level_set_tuning,
 * the tiles the next launch uses), so no device is needed.  Each box is cut
 * into tiles and z-runs of at most tile_z planes.  The class's tile covers
 * the box where a whole one fits; the width left at the box's high x end is
 * covered by narrower, taller tiles (width halved while it does not fit,
 * down to 8, only the last reaching past the box; or one tile of the
 * narrowest width that holds the rest, when that takes fewer tiles over the
 * box's rows), and the last band of
 * rows under the full-width tiles, when at most half a tile tall, by wider,
 * flatter ones (up to 64 wide, each as wide as fits, down to the class's
 * tile); every tile is tile_x x 512 / tile_x points.  A column of tiles at an x
 * face whose ghosts the warp-specialised passes read from the box that owns
 * them splits its z extent first where that owner changes, so that no item
 * reads such a ghost row from two boxes.  The order is by the place of the
 * tile in its domain (domain, then z, y, x of its first point).  Errors:
 * SC_EINVAL for NULL n, or NULL out with cap > 0. */
int sc_level_work_items(const sc_level* level, int32_t* out, int64_t cap, int64_t* n);

/* Run-time tuning of the batched stencil kernels (GPU counterpart of the
 * paper's random-restart hill climbing, Sec. 3.2): for every size class,
 * times candidate tiles on scratch fields of this level (in the launch of
 * the whole level), moves to better neighbours, restarts at random with
 * small probability, aborts candidates that run longer than `abort_factor`
 * x the best time, and keeps the best.  Unless sc_level_set_fusion fixed
 * the form, it does so for one and for two RK4 stages per pass and keeps
 * the form whose step is faster (selecting between sets of loop kernels,
 * Sec. 3.3); for the one-stage form it also times both stagings of its raw
 * inputs (sc_level_set_staging) with the tuned tiles, unless fixed.
 * budget_ms bounds the total tuning time.  Results are applied
 * to the level and, if cache_path is not NULL, merged into that on-disk
 * cache (keyed by GPU name, SM count, arithmetic, form and class extent)
 * and reused from it; a cache line whose tile sc_level_set_tuning would
 * reject is ignored.  Synchronises the stream. */
int sc_level_autotune(sc_level* level, int32_t seed, double budget_ms,
                      double abort_factor, const char* cache_path, void* stream);

/* ---- kernels ----------------------------------------------------------- */

/* Fill the ghost points of `field` from the owners' interior points
 * (bit-exact copies), every box of the level, one batched launch.
 * Ghosts with no owner (outside a non-periodic domain face) are untouched. */
int sc_level_fill_ghosts(sc_level* level, double* field, void* stream);

/* out = L u on every interior point (ghosts of u must be filled, e.g. by
 * sc_level_fill_ghosts).  Ghost and padding entries of out are untouched.
 * u and out must not overlap. */
int sc_level_apply_laplacian(sc_level* level, const double* u, double* out,
                             void* stream);

/* Advance (u, pi) by nsteps classic RK4 steps of dt, in place.  dt points to
 * ndt host doubles: ndt == 1 (one step size) or ndt == number of domains
 * (step size of each domain).  c2 is read on interior points only.  The
 * ghosts of every stencil input are gathered before the pass that reads it
 * (one batched launch, inside the step's CUDA graph in SC_MODE_GRAPH), so on
 * return the ghosts of u hold the input of the last pass, not the result.
 * The warp-specialised two-stage passes read the two-point-wide x-face
 * ghosts that another box of the level owns (even x extents, 16-byte
 * aligned rows) from that box directly; those ghosts are not gathered and
 * keep older values.
 * A box that alone tiles a domain periodic on every axis, with an even x
 * extent and x, y extents >= 2 (a self-periodic box), is an exception: the
 * kernels read the periodic images of its interior for its x and y ghosts,
 * which are not written, and only its z ghosts are gathered; the
 * warp-specialised two-stage passes (SC_PASS_WARP_SPECIALISED) read its z
 * ghosts the same way when its z extent is >= 2, and gather nothing for it.
 * SC_MODE_PER_BOX gathers the same ghosts as the other modes, one launch per
 * box; with the one-role pass kernels (SC_PASS_ONE_ROLE) it gathers every
 * ghost.  sc_level_fill_ghosts always fills every ghost.
 * mode is one of SC_MODE_*.  Scratch stage arrays are allocated on the first
 * call.
 * A level with a domain that is not periodic on every axis takes ONE step
 * per call (SC_EINVAL for nsteps > 1).  Before each call the caller writes
 * boundary data into the ghosts of u and pi that no box owns; they are held
 * over the step.  Ghosts that a box owns are filled by the exchange, and
 * every star ghost value of u and pi must be finite.  Later stages see zeros
 * in the unowned ghosts, so after the step the interior points within 4 of
 * such a face are boundary-influenced and the rest equal the exact step's
 * (the refinement hierarchy's buffer zone, include/sc_hierarchy.h). */
int sc_level_rk4_step(sc_level* level, double* u, double* pi, const double* c2,
                      const double* dt, int32_t ndt, int32_t nsteps, int32_t mode,
                      void* stream);

/* Same step, end to end from HOST memory: copies u, pi, c2 (host, ideally
 * pinned) to library-owned device buffers, runs nsteps steps, and copies
 * the results to u_out, pi_out (host).  Synchronises the stream. */
int sc_level_rk4_step_host(sc_level* level, const double* u, const double* pi,
                           const double* c2, double* u_out, double* pi_out,
                           const double* dt, int32_t ndt, int32_t nsteps,
                           void* stream);

/* Misfit loss L = 1/2 sum_interior (u - u_obs)^2 h^3 (h per domain) into
 * *loss (DEVICE double), and, if seed != NULL, seed = h^3 (u - u_obs) on
 * interior points (the adjoint seed dL/du).  Deterministic reduction. */
int sc_level_misfit(sc_level* level, const double* u, const double* u_obs,
                    double* loss, double* seed, void* stream);

/* Forward pass for differentiation: runs nsteps RK4 steps from (u0, pi0)
 * (batched launches; with one stage per pass the ghosts of each stage
 * output are written by the stage kernel itself, from the level's exchange
 * list grouped by source box and face slab, so u_T's ghosts are filled --
 * for a self-periodic box (see sc_level_rk4_step) its z ghosts only;
 * with two stages per pass they are gathered before each pass and u_T's
 * ghosts are not refreshed), keeping the state every ckpt_every steps in
 * library-owned checkpoint fields (the level's tape, replacing any earlier
 * tape), and writes the final state to u_T, pi_T (either may be NULL).
 * Inputs are not modified.  Requires periodic domains.  Device memory:
 * 2 * ceil(nsteps / ckpt_every) fields for the tape. */
int sc_level_forward_tape(sc_level* level, const double* u0, const double* pi0,
                          const double* c2, const double* dt, int32_t ndt,
                          int32_t nsteps, int32_t ckpt_every, double* u_T,
                          double* pi_T, void* stream);

/* Reverse sweep over the tape (adjoint method).  Given the adjoint seeds
 * gu_T, gpi_T = dLoss/d(u_T, pi_T) (interior values; NULL means zero),
 * writes g_u0, g_pi0 = dLoss/d(u0, pi0) and g_c2 = dLoss/dc2 on interior
 * points.  Each segment between checkpoints is recomputed forward, recording
 * L w.u of every stage (4 * ckpt_every fields), then reversed step by step.
 * The adjoint stage applies A^T(a, b) = (L(c2 * b), a) -- c2 multiplies the
 * adjoint variable before the symmetric stencil -- in reverse stage order.
 * c2 must be the pointer (and values) given to sc_level_forward_tape.
 * SC_EINVAL if there is no tape. */
int sc_level_backward_tape(sc_level* level, const double* c2, const double* gu_T,
                           const double* gpi_T, double* g_u0, double* g_pi0,
                           double* g_c2, void* stream);

/* sc_level_forward_tape followed by sc_level_backward_tape, for seeds that
 * do not depend on the final state (u_T / pi_T may be NULL). */
int sc_level_grad(sc_level* level, const double* u0, const double* pi0,
                  const double* c2, const double* dt, int32_t ndt, int32_t nsteps,
                  int32_t ckpt_every, const double* gu_T, const double* gpi_T,
                  double* g_u0, double* g_pi0, double* g_c2, double* u_T,
                  double* pi_T, void* stream);

/* Wait for the stream and report any device error word (SC_EDEVICE). */
int sc_level_sync(sc_level* level, void* stream);

/* Kernel kinds for per-kernel timing. */
#define SC_KERNEL_STAGE 0        /* forward stage kernel                     */
#define SC_KERNEL_GATHER 1       /* ghost gather                             */
#define SC_KERNEL_STAGE_RECORD 2 /* forward stage kernel recording L w.u     */
#define SC_KERNEL_ADJ_A 3        /* adjoint pass 1: L(c2 .) twice, c2 products */
#define SC_KERNEL_ADJ_B 4        /* adjoint pass 2: L(c2 .) twice              */
#define SC_KERNEL_ADJ_C 5        /* adjoint: pointwise combination           */
#define SC_KERNEL_PAIR_A 6       /* two-stage pass A (stages 1, 2)           */
#define SC_KERNEL_PAIR_B 7       /* two-stage pass B (stages 3, 4)           */

/* Per-kernel device times of the last timed call: sc_level_rk4_step with
 * SC_MODE_TIMED, or sc_level_forward_tape / sc_level_backward_tape while
 * profiling is on.  Each launch of those calls is bracketed by CUDA events
 * on the stream; these return the summed durations and launch counts of one
 * kernel kind (SC_KERNEL_*), or of the stage kernel and the gather.  Wait
 * for those events. */
int sc_level_kernel_time(sc_level* level, int32_t kind, double* ms, int64_t* launches);
int sc_level_kernel_times(sc_level* level, double* stage_ms, int64_t* stage_launches,
                          double* gather_ms, int64_t* gather_launches);

/* Time every launch of later sc_level_forward_tape / sc_level_backward_tape
 * calls with CUDA events (on != 0) or not (0, the default). */
int sc_level_set_profiling(sc_level* level, int32_t on);

/* Number of kernel launches the library enqueued since creation (graph
 * launches count their kernel nodes).  For measurement bookkeeping. */
int sc_level_launch_count(const sc_level* level, int64_t* n);

/* ---- RK4 without device allocation --------------------------------------
 * The paper has no counterpart of this entry point.  It serves callers that
 * cannot allocate device memory (for example while their own allocator owns
 * the whole device, or where cudaMalloc/cudaFree are forbidden after
 * start-up): it advances ONE periodic box by nsteps RK4 steps (FP64 form of
 * the stage kernel, same results as sc_level_rk4_step with SC_ARITH_FP64
 * and one stage per pass on a one-box periodic level) and calls no
 * cudaMalloc, cudaFree or other
 * allocating routine.  Its four stage arrays live in a file-scope static
 * device array of 16 MiB (4 arrays of 2^19 doubles) that every GPU loading
 * the library holds until the process exits.
 *  - u, pi, c2: caller-owned DEVICE pointers, 16-byte aligned, each pointing
 *    at the first element (ghost corner (-2,-2,-2)) of one padded box laid
 *    out as in the level layout: row pitch py = roundup(nx+4, 16), plane
 *    pitch pz = py*(ny+4), (nz+4) planes.  u and pi are updated in place;
 *    their ghosts are refreshed internally; c2 is read on interior points.
 *  - h: grid spacing; dt: step; nsteps >= 0.
 *  - Boxes whose padded size pz*(nz+4) exceeds 2^19 doubles are rejected
 *    with SC_EINVAL ("box too large"; the size is formed in 64 bits, so no
 *    extent can wrap it), as are bad pointers or sizes, before any CUDA
 *    call.  A CUDA error already pending from earlier work is returned as
 *    SC_ECUDA before anything is enqueued; a failed launch stops the call
 *    at that launch (SC_ECUDA).
 *  - There is no device error word: this FP64 path has no fixed-point
 *    scale or non-finite check to report, so a non-finite input simply
 *    propagates into the results, as FP64 arithmetic does.
 *  - The first call on a device resolves the static array's device address
 *    (cudaGetSymbolAddress, with that device current); make that first call
 *    before any stream capture on the device.
 *  - Every call shares the one array and leaves the last call's contents in
 *    it (nothing there needs to start at zero); calls whose work overlaps on
 *    the GPU race with each other. */
int sc_box_rk4_step_noalloc(double* u, double* pi, const double* c2, int32_t nx,
                            int32_t ny, int32_t nz, double h, double dt, int32_t nsteps,
                            void* stream);

/* Message of the last failing call on this thread ("" if none). */
const char* sc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SC_LEVEL_H */
