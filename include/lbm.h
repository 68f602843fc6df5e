/*
 * lbm.h -- C ABI of the GB300 MinxEnt-LBM library (liblbm.so).
 *
 * The library advances lattice Boltzmann simulations with the MinxEnt
 * collision of Wilson, Pugh & Dawson, "Stabilization of the Lattice Boltzmann
 * Method Using Information Theory" (arXiv:1801.03863), on one CUDA GPU.
 * One time step is the paper's Eq. (2): a local collision followed by
 * streaming along the lattice velocities, with the boundary rules of
 * Sec. IV.F.  The library runs it as one fused pull-stream + collide +
 * boundary pass per step.
 *
 * Conventions for every entry point:
 *  - Return value: LBM_OK (0) or a negative LBM_ERR_* code;
 *    lbm_status_string() names it.  A CUDA failure inside a call returns
 *    LBM_ERR_CUDA and leaves the context usable only for lbm_destroy().
 *  - Host arrays are caller-owned, FP64, row-major [y][x] with x fastest;
 *    ensembles concatenate their instances in creation order.  The library
 *    keeps no pointer to them after the call returns.
 *  - Device populations are owned by the context (in the block the caller
 *    passed through lbm_opts.device_mem, or allocated by the library).
 *  - Calls on one context are not thread-safe; separate contexts are
 *    independent.  Work is issued on lbm_opts.stream.
 *  - The populations are stored as deviations f_a - W_a rho0 (SoA, one plane
 *    per velocity, rows padded to a multiple of 8 nodes).
 */
#ifndef LBM_H
#define LBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque context owned by the library. */
typedef struct lbm_ctx lbm_ctx;

/* Return codes. */
#define LBM_OK 0
#define LBM_ERR_ARG (-1)      /* invalid argument (null pointer, size, enum)   */
#define LBM_ERR_ALLOC (-2)    /* device memory could not be obtained           */
#define LBM_ERR_CUDA (-3)     /* a CUDA runtime call failed                    */
#define LBM_ERR_UNSTABLE (-4) /* some post-collision population was negative or
                                 not finite (Sec. IV.H's stability criterion);
                                 sticky, reported by lbm_moments / lbm_status */
#define LBM_ERR_STATE (-5)    /* call out of order (e.g. step before init)     */
#define LBM_ERR_NODEV (-6)    /* no CUDA device, or not an sm_103 device       */
#define LBM_ERR_TIMEOUT (-7)  /* a bounded device-side wait on an asynchronous
                                 copy ran out; the step's outputs are invalid
                                 (sticky, reported by lbm_status / lbm_moments).
                                 Test hooks, read at context creation: the
                                 environment variable LBM_SPIN_LIMIT (1 .. 2^20)
                                 shortens the waits, LBM_TEST_LOST_TILE = t makes
                                 the TMA-staged kernel skip the copies of tile t,
                                 so that its waits run out without any fault */

/* Lattices: D2Q9 of Table I; D1Q3, its one-dimensional restriction
 * (velocities 0, +1, -1; weights 2/3, 1/6, 1/6). */
typedef enum { LBM_D1Q3 = 1, LBM_D2Q9 = 2 } lbm_lattice;

/* Boundaries (Sec. IV.F).
 *  PERIODIC       every direction wraps.
 *  ZERO_GRADIENT  x ends copy the end node's own post-collision populations
 *                 into the ghost beyond it (so a population entering at an
 *                 end equals the one that left it, same direction); y wraps.
 *  CAVITY         D2Q9 lid-driven cavity: the outer ring x = 0, x = nx-1,
 *                 y = 0 (and both top corners) are full-way bounce-back walls;
 *                 the top row y = ny-1 strictly between the corners is the
 *                 moving lid, set every step to f^eq(rho0, (u_lid, 0)). */
typedef enum { LBM_BC_PERIODIC = 0, LBM_BC_ZERO_GRADIENT = 1, LBM_BC_CAVITY = 2 } lbm_bc;

/* Collision rules.
 *  MINXENT4  Sec. IV.C-E: minimise the discrete KLD (Eq. discrete_KLD) under
 *            mass, momentum and the two viscous-stress constraints (Eqs.
 *            discreteprobconst .. discreteisoconst), one Newton-Raphson step
 *            in moment space from the equilibrium moments.  On D1Q3 the three
 *            constraints fix the populations and the rule equals BGK.
 *  SRT       Eq. (bgkcollision) with the polynomial equilibrium
 *            (Eq. numerical-plyeqm); the bandwidth reference kernel.
 *  MINXENT2  Sec. IV.C-E with two free moments (M2, M3) and the extra
 *            heat-flux constraints of Eqs. (extraconstraint1/2), relaxed at
 *            1/tau2 (Eq. tau2).
 *  MRT       Eq. (mrtcollision) with Table III's MRT-LBM rates
 *            diag(0, 1.64, 1.54, 0, 1/tau2, 0, 1/tau2, 1/tau, 1/tau).
 *  TRT       Eq. (mrtcollision) with Table III's TRT-LBM rates
 *            diag(0, 1/tau, 1/tau, 0, 1/tau2, 0, 1/tau2, 1/tau, 1/tau).
 * On D1Q3 every rule relaxes the one non-conserved moment at 1/tau: BGK. */
typedef enum {
    LBM_MINXENT4 = 0,
    LBM_SRT = 1,
    LBM_MINXENT2 = 2,
    LBM_MRT = 3,
    LBM_TRT = 4
} lbm_collision;

/* Reading of Eq. (tau2) for the heat-flux rate 1/tau2 (MINXENT2, MRT, TRT).
 *  PRINTED  tau2 = (8 tau - 1) / (2 tau - 1), as printed.
 *  MAGIC    tau2 = (8 tau - 1) / (8 (2 tau - 1)), the form that gives the
 *           TRT "magic" product (tau - 1/2)(tau2 - 1/2) = 3/16 of the
 *           relation the paper cites; the printed form may lack the 8. */
typedef enum { LBM_TAU2_PRINTED = 0, LBM_TAU2_MAGIC = 1 } lbm_tau2_reading;

/* Arithmetic / storage types.  compute = LBM_F64 requires storage = LBM_F64;
 * compute = LBM_F32 allows storage LBM_F32, LBM_F16 or LBM_BF16. */
typedef enum { LBM_F64 = 0, LBM_F32 = 1, LBM_F16 = 2, LBM_BF16 = 3 } lbm_dtype;

typedef struct {
    int32_t compute;           /* lbm_dtype of the collision arithmetic (default F64) */
    int32_t storage;           /* lbm_dtype of the stored deviations (default F64)    */
    int32_t collision;         /* lbm_collision (default MINXENT4)                   */
    int32_t autotune;          /* 1: time candidate launch shapes at create (default 1) */
    double rho0;               /* reference density of the deviation storage and of
                                  the lid equilibrium (default 1.0)                  */
    void* stream;              /* cudaStream_t for all work; NULL = default stream   */
    void* device_mem;          /* optional caller-owned device block (>= 256-byte
                                  aligned) of lbm_required_bytes() bytes; NULL = the
                                  library allocates and frees its own                */
    uint64_t device_mem_bytes; /* size of device_mem                                */
    int32_t tau2_reading;      /* lbm_tau2_reading (default PRINTED)                 */
    int32_t reserved;          /* must be 0                                         */
} lbm_opts;

/* Fill *opts with the defaults listed above. */
void lbm_default_opts(lbm_opts* opts);

/* Device bytes a context of this shape needs (populations, both time levels,
 * tables, status words, reduction partials and an FP64 staging area).
 * dims: count*2 int64 (nx, ny) per instance; D1Q3 requires ny == 1. */
int lbm_required_bytes(lbm_lattice lat, int32_t count, const int64_t* dims,
                       const lbm_opts* opts, uint64_t* bytes);

/* Create one lattice of dims[0] x dims[1] nodes (D1Q3: dims[1] == 1) with
 * kinematic viscosity nu > 0 in lattice units.  tau = 3 nu + 1/2 follows
 * from Eq. (visco-tau) with dx = dt = 1.  u_lid is used by LBM_BC_CAVITY
 * only.  opts may be NULL (defaults).  *out receives the context. */
int lbm_create(lbm_ctx** out, lbm_lattice lat, const int64_t* dims, double nu, lbm_bc bc,
               double u_lid, const lbm_opts* opts);

/* Create an ensemble of count independent lattices that share lattice,
 * boundary kind and opts but not size (dims: count*2), viscosity (nu:
 * count) or lid speed (u_lid: count, may be NULL).  One step advances every
 * instance in a single persistent launch over a per-instance tile table. */
int lbm_create_batch(lbm_ctx** out, lbm_lattice lat, int32_t count, const int64_t* dims,
                     const double* nu, const double* u_lid, lbm_bc bc, const lbm_opts* opts);

/* Initial populations at equilibrium (Sec. IV.F) from host FP64 fields
 * rho, ux, uy (each sum(nx*ny) long, instances concatenated); ux/uy may be
 * NULL for zero; uy is ignored on D1Q3.  Resets the status counters.
 * Page-locked host arrays (cudaHostAlloc, cudaHostRegister) are read in
 * place by the initialising kernel; other host memory is first copied to a
 * device staging area.  Synchronises. */
int lbm_init(lbm_ctx* ctx, const double* rho, const double* ux, const double* uy);

/* Same as lbm_init with DEVICE pointers, ordered on the context's stream;
 * does not synchronise. */
int lbm_init_device(lbm_ctx* ctx, const double* rho, const double* ux, const double* uy);

/* Initial populations of ONE instance of an ensemble at equilibrium
 * (Sec. IV.F: f = f^eq(rho, u), Eq. numerical-plyeqm) from host FP64 fields
 * of that instance alone (nx*ny values each, [y][x]; ux/uy may be NULL for
 * zero; uy is ignored on D1Q3).  The other instances are left untouched and
 * the instance's status counters are reset.  Allowed before the first step
 * after context creation, lbm_init or lbm_set_populations (LBM_ERR_STATE
 * once the context has stepped: the stored field is then post-collision).
 * The context counts as initialised once every instance has been set, by
 * this call or by lbm_init.  Synchronises. */
int lbm_init_batch(lbm_ctx* ctx, int32_t instance, const double* rho, const double* ux,
                   const double* uy);

/* Advance every instance by n >= 0 time steps (Eq. 2).  Asynchronous on the
 * context's stream; runs of 16 or more steps replay CUDA graphs of 16
 * launches, captured and uploaded when the context is created. */
int lbm_step(lbm_ctx* ctx, int64_t n);

/* Density and velocity of f(x, t_n) (Sec. II.A: rho = sum f, rho u = sum f v)
 * into host FP64 arrays (sum(nx*ny) each; ux/uy may be NULL).  Synchronises
 * the stream; returns LBM_ERR_UNSTABLE if any instance has flagged an
 * unstable node since lbm_init (the fields are written all the same).
 * Page-locked host arrays are written in place by the moments kernel. */
int lbm_moments(lbm_ctx* ctx, double* rho, double* ux, double* uy);

/* lbm_moments into DEVICE FP64 arrays, ordered on the stream, no sync and
 * no status check. */
int lbm_moments_device(lbm_ctx* ctx, double* rho, double* ux, double* uy);

/* Density and velocity of f(x, t_n) (Sec. II.A) of ONE instance into host
 * FP64 arrays of nx*ny values ([y][x]; ux/uy may be NULL): the same values
 * lbm_moments writes for that instance, without reading back the others.
 * Synchronises; returns LBM_ERR_UNSTABLE if this instance has flagged an
 * unstable node since it was initialised (fields written all the same). */
int lbm_moments_batch(lbm_ctx* ctx, int32_t instance, double* rho, double* ux, double* uy);

/* lbm_moments_batch into DEVICE FP64 arrays of nx*ny values, ordered on the
 * stream, no sync and no status check. */
int lbm_moments_batch_device(lbm_ctx* ctx, int32_t instance, double* rho, double* ux,
                             double* uy);

/* Stream function of f(x, t_n) for the lid-driven cavity analysis of
 * Sec. IV.I: per row of every instance, psi(x, y) = - integral from x = 0 to
 * x of u_y dx, in lattice units (node spacing 1, psi = 0 at x = 0), with the
 * composite Simpson rule over pairs of unit intervals and the trapezoidal
 * rule on a last odd interval.  psi: host FP64 array of sum(nx*ny) values in
 * the order of lbm_moments (per instance [y][x]).  D2Q9 only (LBM_ERR_ARG
 * otherwise).  Synchronises; status as lbm_moments.  Normalise by
 * |u_lid| (side - 1) for the paper's psi-hat. */
int lbm_stream_function(lbm_ctx* ctx, double* psi);

/* lbm_stream_function into a DEVICE FP64 array, ordered on the stream, no
 * sync and no status check (uses the context's staging area for u). */
int lbm_stream_function_device(lbm_ctx* ctx, double* psi);

/* lbm_stream_function of ONE instance (Sec. IV.I) into a host FP64 array
 * of nx*ny values; the same values lbm_stream_function writes for that
 * instance.  Synchronises; status as lbm_moments_batch. */
int lbm_stream_function_batch(lbm_ctx* ctx, int32_t instance, double* psi);

/* Populations f(x, t_n) to / from host FP64, layout per instance
 * [a][y][x] (a in the order rest, +x, +y, -x, -y, (+x,+y), (-x,+y),
 * (-x,-y), (+x,-y) for D2Q9; rest, +x, -x for D1Q3), instances
 * concatenated.  set_populations replaces the state; the next step collides
 * the loaded f(x, t_n) in place with the step kernels' arithmetic, so a
 * state read with get_populations and set into another context continues
 * bit for bit when its FP64 values round-trip exactly (always for FP16 and
 * BF16 storage; FP32 and FP64 deviations far below W_a rho0 lose bits in
 * f = W_a rho0 + d -- lbm_save_state / lbm_load_state are exact for every
 * storage type). */
int lbm_get_populations(lbm_ctx* ctx, double* f);
int lbm_set_populations(lbm_ctx* ctx, const double* f);

/* Exact checkpoint / resume.  The paper has no counterpart (a run of Eq. 2
 * is a sequence of states; this saves one and continues from it).
 * lbm_save_state copies the context's state -- the stored population
 * deviations in the storage type and padded layout, whether they are
 * post-collision, the step count and the status counters -- into a host
 * buffer of lbm_state_bytes() bytes; lbm_load_state restores it into a
 * context created with the same lattice, storage type and instance sizes
 * (LBM_ERR_ARG otherwise; collision rule, viscosities and lid speeds may
 * differ).  A loaded context continues bit for bit like the one saved,
 * whatever the storage type.  Both synchronise. */
int lbm_state_bytes(lbm_ctx* ctx, uint64_t* bytes);
int lbm_save_state(lbm_ctx* ctx, void* host_buf);
int lbm_load_state(lbm_ctx* ctx, const void* host_buf);

/* Per-instance totals of f(x, t_n) in FP64 -- out[3*i + 0..2] = sum rho,
 * sum rho u_x, sum rho u_y -- from a deterministic two-pass reduction
 * (fixed summation order, bitwise reproducible).  Host output; syncs. */
int lbm_conservation(lbm_ctx* ctx, double* out);

/* lbm_conservation into a DEVICE FP64 array of 3*count doubles, ordered on
 * the stream, no sync (for checkpoints inside a timed step loop). */
int lbm_conservation_device(lbm_ctx* ctx, double* out);

/* lbm_conservation_device for callers that cannot allocate device memory
 * (an application that owns every allocation through its own pool, a
 * real-time loop that must not hit the allocator's synchronisation, a plugin
 * whose host forbids new allocations).  The paper has no counterpart; this is
 * an interface convenience.  The call allocates nothing: the reduction's
 * scratch is a fixed array inside the library (6 MiB per device, kept until
 * the process exits), enough for contexts of up to 4096 instances; larger
 * contexts get LBM_ERR_ARG.  out: DEVICE pointer to 3*count doubles, same
 * values as lbm_conservation_device.  The first call on a device looks up the
 * array's device address; make that first call outside any CUDA stream
 * capture.  All calls in the process share the array, so calls whose work
 * overlaps on the GPU (different streams, different contexts) race: order
 * them on one stream or synchronise between them.  Ordered on the context's
 * stream; no sync. */
int lbm_conservation_noalloc(lbm_ctx* ctx, double* out);

/* Status counters summed over all instances since lbm_init:
 * counters[0] = nodes whose Newton step was skipped because some start
 * probability was <= 0 (the log of Eq. discrete_KLD is undefined there; the
 * node keeps the constraint-satisfying start point), counters[1] = nodes
 * with a negative or non-finite post-collision population, counters[2] =
 * time steps taken.  Syncs.  Per-instance: lbm_status_instance. */
int lbm_status(lbm_ctx* ctx, int64_t* counters);
int lbm_status_instance(lbm_ctx* ctx, int32_t instance, int64_t* counters);

/* Launch shape in use: out[0] = nodes per thread, out[1] = tile width in
 * thread chunks, out[2] = tile height in rows, out[3] = grid size (CTAs),
 * out[4] = kernel kind (0: register-chunk kernel; 1 to 4: the TMA-staged
 * D2Q9 kernel, whose CTAs have one warp that only moves tiles in and out
 * besides the colliding warps.  1: large tiles, 8-warp CTAs, 1792 nodes for
 * 2-byte storage or 896 for FP32, two-stage ring; 2: small tiles, 8-warp
 * CTAs, 896 / 448 nodes, three-stage ring; 3: 10-warp CTAs, 2304 / 1152
 * nodes, two-stage ring; 4: deep ring, one 16-warp CTA per SM, 1920 / 960
 * nodes, five stages (four for FP32 storage).  For kinds 1
 * to 4 the tile width is 64/128/256 nodes chosen per instance (at most
 * 32 tile nodes / colliding threads; of those, for the MinxEnt rules the
 * one whose tiles cover the instance with the fewest padding nodes, for the
 * others the widest) and out[1], out[2] are 0;
 * tiles go in and out of
 * shared memory by TMA).  Selection: the create-time
 * autotuner (each candidate shape timed over back-to-back launches, the
 * candidates within 5 % of the fastest timed again as a captured graph,
 * which decides; the choice
 * is cached per device, lattice, types, rule, boundary and instance sizes
 * for the life of the process, and in the text file named by the
 * environment variable LBM_AUTOTUNE_CACHE when set, which later processes
 * reuse without timing), or the environment variable LBM_SHAPE = "V,tw,th"
 * (register chunks), "smem" (kind 1), "smems" (kind 2), "smemw" (kind 3) or
 * "smemd" (kind 4). */
int lbm_launch_shape(lbm_ctx* ctx, int32_t* out);

/* Destroy a context (NULL-safe).  Frees library-owned memory only. */
int lbm_destroy(lbm_ctx* ctx);

/* Static description of a return code. */
const char* lbm_status_string(int code);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
