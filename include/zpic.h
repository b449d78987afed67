/*
 * zpic.h -- C ABI of the GB300 2D3V electromagnetic particle-in-cell step.
 *
 * The method is the PIC cycle of Guidotti et al., "Particle-In-Cell
 * Simulation using Asynchronous Tasking" (arXiv 2106.12485), Sec. 2.2:
 *   (1) bilinear interpolation of E, B at each particle,
 *   (2) leapfrog + relativistic Boris push,
 *   (3) exact charge-conserving (Villasenor-Buneman) current deposition,
 *   (4) Yee-mesh FDTD advance of E, B with the current just deposited,
 * with the spatial decomposition of Sec. 3.2 (regions with ghost cells,
 * particles handed to neighbours, at most one cell moved per step) done
 * here as 2D tiles on the GPU, and the laser initialisation and moving
 * window of Sec. 4.1 (LWFA).
 *
 * Units: normalised, c = 1, time in 1/w_p, length in c/w_p, E and B in
 * m c w_p / e, momenta u = gamma v.  dB/dt = -curl E, dE/dt = curl B - J.
 *
 * Grid: nx*ny cells of dx = box_x/nx, dy = box_y/ny.  Staggering
 *   Ex(i+1/2, j)  Ey(i, j+1/2)  Ez(i, j)  Bx(i, j+1/2)  By(i+1/2, j)
 *   Bz(i+1/2, j+1/2); Jx, Jy, Jz co-located with Ex, Ey, Ez.
 * Time centring: x, E, B at integer steps, u at half steps, J at n+1/2.
 * y is periodic; x is periodic or open (moving window).
 *
 * Conventions for every entry point:
 *  - return value: ZPIC_OK (0) or a negative ZPIC_E* code; nothing throws
 *    across the ABI; zpic_strerror() names a code and zpic_last_error()
 *    gives the message of the last failure on the calling thread.
 *  - handles are owned by the library and freed by the matching destroy.
 *  - all buffers passed in are host memory owned by the caller, unless the
 *    argument says "device"; the library copies what it needs and keeps no
 *    pointer to caller memory after the call returns.
 *  - zpic_step is asynchronous on the handle's stream; getters synchronise.
 *  - one host thread at a time per handle.
 *  - the library needs a CUDA device; with none (or without the kernels for
 *    it) every call that would touch the device returns ZPIC_ECUDA.  There
 *    is no CPU fallback.
 */
#ifndef ZPIC_H
#define ZPIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ZPIC_MAX_SPECIES 8
#define ZPIC_VERSION 1

/* status codes */
#define ZPIC_OK 0
#define ZPIC_EINVAL (-1)    /* bad argument, NULL handle or buffer        */
#define ZPIC_ECFL (-2)      /* dt >= 1/sqrt(1/dx^2 + 1/dy^2)              */
#define ZPIC_ENOMEM (-3)    /* device or host allocation failed           */
#define ZPIC_ECUDA (-4)     /* CUDA runtime error / no usable device      */
#define ZPIC_EOVERFLOW (-5) /* particle storage exhausted after resorting */
#define ZPIC_ENAN (-6)      /* non-finite value detected                  */
#define ZPIC_ETIMEOUT (-7)  /* a bounded device wait gave up              */
#define ZPIC_ECAP (-8)      /* destination buffer too small               */
#define ZPIC_ENOTSUP (-9)   /* option not supported by this build         */

/* Errors that end a handle's run (ZPIC_EOVERFLOW after a failed re-sort,
 * ZPIC_ENAN, ZPIC_ETIMEOUT, a corrupted store) are sticky: every later step
 * or sync of that handle returns the same code.
 *
 * Testing hook: the environment variable ZPIC_FAULT (read at every check)
 * injects failures on the host without touching the GPU: "alloc" makes
 * every device allocation fail (ZPIC_ENOMEM), "launch" makes every kernel
 * or graph launch fail before anything is launched (ZPIC_ECUDA from
 * zpic_step; the handle stays usable once the variable is cleared),
 * "timeout" makes zpic_sync report a bounded device wait that gave up
 * (ZPIC_ETIMEOUT, sticky). */

/* precision of fields and particle state */
#define ZPIC_FP32 0
#define ZPIC_FP64 1

/* x boundary (y is always periodic) */
#define ZPIC_BC_PERIODIC 0
#define ZPIC_BC_OPEN 1

/* field selectors */
#define ZPIC_EX 0
#define ZPIC_EY 1
#define ZPIC_EZ 2
#define ZPIC_BX 3
#define ZPIC_BY 4
#define ZPIC_BZ 5
#define ZPIC_JX 6
#define ZPIC_JY 7
#define ZPIC_JZ 8

/* density profiles of the initial load (x in box units, absolute frame) */
#define ZPIC_PROFILE_NONE 0    /* no initial particles                   */
#define ZPIC_PROFILE_UNIFORM 1 /* n0 everywhere                          */
#define ZPIC_PROFILE_SLAB 2    /* n0 for x0 <= x_cell < x1, else 0        */
#define ZPIC_PROFILE_RAMP 3    /* 0 below x0, linear to n0 over length x1,
                                  n0 beyond                               */

/* config flags */
#define ZPIC_TRACK_IDS 1       /* keep a per-particle int32 id (parity)    */
#define ZPIC_FILTER_J 2        /* smooth J before the field update with the
                                  compensated binomial filter (Sec. 2.2
                                  digital filter, Sec. 4.1 LWFA runs): per
                                  axis one (1,2,1)/4 and one (-1,6,-1)/4
                                  pass; the J getters then return the
                                  filtered current */
#define ZPIC_DETERMINISTIC 4   /* bitwise reproducible runs: the current of
                                  a step is an exact integer sum, whatever
                                  order tiles and particles add in, so
                                  fields, currents, particles and field
                                  energies repeat bit for bit (the kinetic
                                  energy records sum per-particle values
                                  in store order and repeat to rounding).
                                  FP32 always works this way (this flag
                                  changes nothing); FP64 then sums J as
                                  64-bit fixed point in units of 2^-47 of
                                  the largest one-segment contribution
                                  (range 2^16 such units per value and
                                  step) instead of double atomics */

typedef struct {
    double q_over_m;    /* charge-to-mass ratio (electrons: -1)          */
    int ppc_x, ppc_y;   /* particles per cell at density n0              */
    int lattice;        /* 1: offsets (k+1/2)/ppc; 0: uniform random     */
    double u_th[3];     /* thermal spread of u per axis                  */
    double u_fl[3];     /* drift of u                                    */
    int profile;        /* ZPIC_PROFILE_*                                */
    double x0, x1;      /* profile parameters (see above)                */
    double n0;          /* density; a particle carries q = sign(q/m)*w/ppc
                           with weight w = local density                 */
} zpic_species;

typedef struct {
    int enabled;
    double a0;          /* normalised vector potential                   */
    double omega0;      /* laser frequency (units of w_p)                */
    double w0;          /* transverse waist: exp(-(y-yc)^2/w0^2) in field */
    double fwhm;        /* intensity FWHM along x                        */
    double x0;          /* pulse centre in x                             */
    double y_center;    /* pulse axis in y                               */
} zpic_laser;

typedef struct {
    int nx, ny;                 /* cells                                  */
    double box_x, box_y;        /* box size                               */
    double dt;                  /* time step (CFL checked)                */
    int precision;              /* ZPIC_FP32 or ZPIC_FP64                 */
    int bc_x;                   /* ZPIC_BC_PERIODIC or ZPIC_BC_OPEN       */
    int moving_window;          /* 1: window moves at c along +x (needs
                                   bc_x = ZPIC_BC_OPEN)                   */
    int n_species;              /* 0..ZPIC_MAX_SPECIES                    */
    zpic_species species[ZPIC_MAX_SPECIES];
    zpic_laser laser;
    uint64_t seed;              /* generator seed of the initial load     */
    int sim_index;              /* generator stream of this simulation    */
    int energy_every;           /* record energies every k steps; 0: off  */
    int tile_x, tile_y;         /* tile size in cells, 2..32; 0: the size
                                   zpic_autotune chose for this
                                   configuration's class, else 16         */
    int flags;                  /* ZPIC_TRACK_IDS | ZPIC_FILTER_J |
                                   ZPIC_DETERMINISTIC                     */
    double capacity_slack;      /* spare tile capacity fraction; 0: 0.25  */
    int sort_every;             /* re-sort every tile's particles into
                                   cell-interleaved order every k steps
                                   (k >= 1); -1: never; 0: the interval
                                   zpic_autotune chose for this
                                   configuration's class, else never      */
    int push_ctas_per_sm;       /* resident particle-kernel CTAs per SM
                                   (1..8, capped at what fits); 0: the
                                   number zpic_autotune chose for this
                                   configuration's class, else all that
                                   fit                                     */
} zpic_config;

/* Particle arrays for get/set.  Real arrays (x .. w) hold float when
 * precision == ZPIC_FP32, double when ZPIC_FP64 (the library converts if
 * this differs from the simulation's precision).  Offsets x, y in [0, 1)
 * within cell (ix, iy). */
typedef struct {
    int precision;
    size_t cap;         /* capacity of each array (get)                  */
    size_t n;           /* number of particles (set: supplied, get: out) */
    int32_t *ix, *iy;
    void *x, *y, *ux, *uy, *uz;
    void *w;            /* may be NULL (get: skipped; set: weight 1)     */
    int32_t *id;        /* may be NULL (get: skipped; set: ids 0..n-1)   */
} zpic_particles;

/* One energy record: step k means fields at step k and momenta at k-1/2
 * (after the push of step k-1).  wE = 1/2 sum E^2 dx dy, wB likewise,
 * kin[s] = sum m_p (gamma - 1) dx dy. */
typedef struct {
    int32_t step;
    int32_t n_species;
    double wE, wB;
    double kin[ZPIC_MAX_SPECIES];
} zpic_energy_rec;

/* Forms of the particle kernel (zpic_info.push_variants, one bit each):
 * the 16x16-tile FP32 kernel is compiled separately for species that store
 * neither weights nor ids (the plain layout), with a periodic or an open x
 * boundary; every other species runs the form that reads its layout at run
 * time. */
#define ZPIC_PUSH_GENERIC 1
#define ZPIC_PUSH_PLAIN_PERIODIC 2
#define ZPIC_PUSH_PLAIN_OPEN 4

/* Layout and state summary of a simulation. */
typedef struct {
    int nx, ny, ld;             /* ld = padded row length of field arrays */
    double dx, dy, dt;
    int tile_x, tile_y, ntiles_x, ntiles_y;
    int precision;
    int32_t step;               /* completed steps                        */
    int32_t n_shift;            /* moving-window shifts so far            */
    int n_species;
    int64_t n_particles[ZPIC_MAX_SPECIES];
    int64_t capacity[ZPIC_MAX_SPECIES];
    int32_t resorts;            /* full re-sorts done (overflow recovery)  */
    size_t device_bytes;        /* device memory held                     */
    int32_t push_variants[ZPIC_MAX_SPECIES]; /* ZPIC_PUSH_* bits of the
                                   particle-kernel forms that ran for each
                                   species since creation (recorded by the
                                   kernel itself)                         */
    int32_t sort_every;         /* re-sort interval in use (-1: never)    */
    int32_t push_ctas_per_sm;   /* particle-kernel CTAs per SM in use     */
    int32_t sorts;              /* cell-order re-sorts done on the device */
} zpic_info;

/* Run state beyond fields and particles, for checkpoint / restart. */
typedef struct {
    int64_t step;               /* completed steps                        */
    int32_t n_shift;            /* moving-window shifts done              */
    int32_t reserved;
    int64_t removed[ZPIC_MAX_SPECIES];  /* particles removed at open edges */
} zpic_state;

/* Phase-space quantities for zpic_phasespace. */
#define ZPIC_PS_X 0    /* global x position in cells, ix + x */
#define ZPIC_PS_Y 1    /* global y position in cells, iy + y */
#define ZPIC_PS_UX 2
#define ZPIC_PS_UY 3
#define ZPIC_PS_UZ 4

typedef struct zpic_sim zpic_sim;
typedef struct zpic_batch zpic_batch;

/* Creates a simulation: validates cfg (ZPIC_EINVAL, ZPIC_ECFL), allocates
 * device memory, draws the initial particles on the GPU from the counter-
 * based SplitMix64 stream (seed, sim_index, species) and writes the laser
 * fields (Sec. 4.1).  *out receives the handle.  cfg is copied. */
int zpic_create(const zpic_config *cfg, zpic_sim **out);

/* Frees a simulation created by zpic_create (not a batch view); the
 * device memory of its fields and tile stores goes back to the allocator. */
int zpic_destroy(zpic_sim *sim);

/* Enqueues n time steps on the handle's stream and returns.  One step is
 * the PIC cycle of Sec. 2.2 (Fig. 1): interpolation of E, B at the
 * particles, Boris push, charge-conserving deposition, Yee field advance;
 * then the hand-over of particles that crossed into a neighbouring tile
 * (the region hand-over of Sec. 3.2, at most one cell per step) and the
 * moving-window shift of Sec. 4.1.  Errors of earlier steps found at the
 * last synchronisation are returned here (ZPIC_EOVERFLOW, ZPIC_ENAN,
 * ZPIC_ETIMEOUT sticky; ZPIC_ECUDA on a failed launch). */
int zpic_step(zpic_sim *sim, int n);

/* Waits for all enqueued steps; recovers from tile-capacity overflow by
 * re-sorting with more capacity and re-running the steps that were held
 * back (a tile, like a region of Sec. 3.2, holds the particles of its
 * cells; one that receives more than its room parks them until the host
 * re-sorts).  Returns the device status: ZPIC_OK, or the sticky
 * ZPIC_EOVERFLOW (storage exhausted after re-sorting), ZPIC_ENAN,
 * ZPIC_ETIMEOUT, ZPIC_ECUDA. */
int zpic_sync(zpic_sim *sim);

/* Uses `stream` (a cudaStream_t) for all later work of the handle.  NULL
 * restores the library's own stream.  The caller keeps the stream alive
 * while the handle uses it. */
int zpic_set_stream(zpic_sim *sim, void *stream);

/* Copies the interior nx*ny values of field `which` (ZPIC_EX..ZPIC_JZ),
 * row-major dst[j*nx + i], at the current step.  J is the current of the
 * last step.  cap is the number of elements dst holds (ZPIC_ECAP if less
 * than nx*ny).  _f32 narrows FP64 simulations; _f64 widens FP32 ones. */
int zpic_get_fields_f32(zpic_sim *sim, int which, float *dst, size_t cap);
int zpic_get_fields_f64(zpic_sim *sim, int which, double *dst, size_t cap);

/* Overwrites field `which` (E or B only) with n = nx*ny values. */
int zpic_set_fields_f64(zpic_sim *sim, int which, const double *src,
                        size_t n);

/* Number of particles of a species (synchronises); particles leave only
 * through an open x boundary and enter only with the moving window's new
 * column (Sec. 4.1). */
int zpic_num_particles(zpic_sim *sim, int species, int64_t *n);

/* Copies the particles of a species into dst (tile order): global cell
 * (ix, iy), offsets (x, y) in [0, 1), u = gamma v at the half step of the
 * leapfrog (Sec. 2.2), weight and id when the arrays are given.  The
 * arrays are caller-owned host memory of dst->cap elements; ZPIC_ECAP if
 * that is too small, ZPIC_EINVAL for NULL arrays or a bad species;
 * *n_written receives the count. */
int zpic_get_particles(zpic_sim *sim, int species, const zpic_particles *dst,
                       size_t *n_written);

/* Like zpic_get_particles for the tiles tile_begin <= t < tile_end only
 * (tile t = ty * ntiles_x + tx of zpic_info), in tile order; for reading a
 * region of a large simulation without copying all of it. */
int zpic_get_particles_tiles(zpic_sim *sim, int species, int tile_begin,
                             int tile_end, const zpic_particles *dst,
                             size_t *n_written);

/* Replaces the particles of a species with src (copied to the device and
 * sorted into tiles there).  Particles must have 0 <= ix < nx,
 * 0 <= iy < ny and offsets in [0, 1) (ZPIC_EINVAL otherwise). */
int zpic_set_particles(zpic_sim *sim, int species, const zpic_particles *src);

/* Copies the energy history (one record per energy_every steps): field
 * energies and kinetic energy per species, summed on the device in
 * compensated FP64 (the validation quantity of Sec. 4.2).  dst is
 * caller-owned host memory of cap records; ZPIC_ECAP if too small.  With
 * dst == NULL and cap == 0 only *n_written is set (size query). */
int zpic_energy(zpic_sim *sim, zpic_energy_rec *dst, size_t cap,
                size_t *n_written);

/* Energies of the current fields (synchronises): *wE = 1/2 sum E^2 dx dy,
 * *wB = 1/2 sum B^2 dx dy over the nx*ny cells (Sec. 2.2 fields, the same
 * quantities as zpic_energy_rec).  Per-row partial sums go to scratch
 * memory the simulation allocated at creation.  The rows are summed in a
 * fixed order, so repeated calls give identical results. */
int zpic_field_energy(zpic_sim *sim, double *wE, double *wB);

/* The same energies as zpic_field_energy, for callers that cannot
 * allocate device memory when they need them (real-time loops that must not
 * wait on an allocator, hosts that give the library a fixed memory budget).
 * The paper has no counterpart; this entry point allocates nothing.
 *   ex .. bz: device arrays (FP32) of ny rows of ld >= nx values, owned by
 *             the caller; nx*ny cells of size dx*dy are summed (values in
 *             the ld - nx padding columns are not read).
 *   out:      host array of 2 doubles: 1/2 sum E^2 dx dy, 1/2 sum B^2 dx dy.
 *   stream:   cudaStream_t to run on (NULL: the default stream); the call
 *             returns after the stream has finished the work.
 * Scratch: a static device array built into the library for at most 65536
 * rows (1 MiB + 16 bytes, held by every GPU that loads the library until
 * exit); ny > 65536 returns ZPIC_EINVAL.  The first call on each device
 * (and the first after the device's context changed, e.g. after
 * cudaDeviceReset) looks up that array's address with the device current,
 * so make the first call on a device before capturing any stream.  All
 * calls share the array: calls that overlap on the GPU (different streams,
 * or several host threads) race and may return wrong sums.  Nothing in it
 * needs clearing: each call writes every value it reads.  Errors:
 * ZPIC_EINVAL (NULL pointer, bad sizes), ZPIC_ECUDA (no device, launch or
 * copy failure). */
int zpic_field_energy_noalloc_f32(const float *ex, const float *ey,
                                  const float *ez, const float *bx,
                                  const float *by, const float *bz, int nx,
                                  int ny, int ld, double dx, double dy,
                                  double *out, void *stream);

/* Fills *info (synchronises): grid, tile decomposition (the regions of
 * Sec. 3.2), counts, capacities and the particle-kernel forms that ran.
 * ZPIC_EINVAL for NULL. */
int zpic_get_info(zpic_sim *sim, zpic_info *info);

/* Per-tile particle counts of a species (the regions of Sec. 3.2), tile
 * index ty*ntiles_x + tx, in the order zpic_get_particles writes them.
 * dst: caller-owned, cap >= ntiles (ZPIC_ECAP otherwise). */
int zpic_get_tile_counts(zpic_sim *sim, int species, int32_t *dst,
                         size_t cap);

/* Checkpoint / restart.  A run is fully described by its configuration,
 * the fields E and B (zpic_get_fields_f64 / zpic_set_fields_f64), the
 * particles of every species with their ids (zpic_get_particles /
 * zpic_set_particles) and this state.  zpic_get_state fills *out (after a
 * sync).  zpic_set_state restores it on a handle created from the same
 * configuration, before or after the fields and particles are set (the
 * current field and particle copies follow the step parity); the energy
 * history restarts empty.  Errors: ZPIC_EINVAL for NULL, a negative step
 * or n_shift, a removed count < 0, or a view into a batch of more than one
 * simulation (the step counter is shared by the batch). */
int zpic_get_state(zpic_sim *sim, zpic_state *out);
int zpic_set_state(zpic_sim *sim, const zpic_state *in);

/* Phase-space report (the paper's field / phase-space reports, Sec. 4.1)
 * computed on the device: a 2D histogram of quantities qx, qy (ZPIC_PS_*)
 * of one species, nbx x nby bins over [range[0], range[1]) x
 * [range[2], range[3]), every particle adding its charge magnitude
 * |q0| w (a charge density per bin).  The bin of a value v on an axis with
 * bounds lo, hi and nb bins is floor((v - lo) * (nb / (hi - lo))),
 * evaluated in double; particles outside either range are not counted.
 * dst: caller-owned, nby rows of nbx doubles (cap >= nbx * nby, else
 * ZPIC_ECAP).  Errors: ZPIC_EINVAL for a bad species, quantity, bin count
 * (1..4096 per axis) or range (hi > lo, finite). */
int zpic_phasespace(zpic_sim *sim, int species, int qx, int qy,
                    const double range[4], int nbx, int nby, double *dst,
                    size_t cap);

/* Tile-size autotuner (host).  Times the step of cfg for each candidate
 * tile size (zpic_autotune_candidates lists them as x, y pairs) on a copy
 * reduced to at most 1024 x 1024 cells (same cell size, dt, species,
 * densities and momenta; slab profiles scaled with the box; a ramp, the
 * window plasma and the laser kept at the same distance from the right
 * edge), `steps` steps after 3 warm-up steps, host wall clock, and returns
 * the fastest in *best_tile_x, *best_tile_y.  The choice is kept for the
 * configuration's class (precision, reduced grid, boundary, window, filter,
 * particles per cell and profile of each species) for the life of the
 * process; zpic_create uses it when tile_x = tile_y = 0.  With
 * ms_per_step == NULL a class already tuned returns at once; otherwise the
 * candidates are timed and ms_per_step[k] (k < cap) receives candidate k's
 * ms per step (negative: the candidate could not run).  Errors:
 * ZPIC_EINVAL (NULL cfg or result, steps outside [1, 10000]), the errors of
 * zpic_create for cfg, ZPIC_ECUDA when no candidate ran. */
int zpic_autotune(const zpic_config *cfg, int steps, int *best_tile_x,
                  int *best_tile_y, double *ms_per_step, int cap,
                  int *n_candidates);
/* Writes up to cap candidate tile sizes (x, y pairs) to tile_xy and returns
 * how many candidates there are. */
int zpic_autotune_candidates(int *tile_xy, int cap);

/* Settings of the particle kernel that zpic_autotune_all chooses. */
typedef struct {
    int tile_x, tile_y;         /* tile size (the region of Sec. 3.2)     */
    int push_ctas_per_sm;       /* resident particle-kernel CTAs per SM:
                                   the tiles in flight per SM, the GPU
                                   counterpart of the regions per core of
                                   the over-decomposition study (Sec. 4.3) */
    int sort_every;             /* cell-order re-sort interval, -1: never */
    double ms_per_step;         /* the chosen setting on the reduced copy */
} zpic_tuning;

/* Tunes tile size, resident CTAs per SM and re-sort interval for cfg's
 * class, one after the other, on the reduced copy zpic_autotune uses: the
 * tile candidates of zpic_autotune_candidates at `steps` timed steps, then
 * 1..3 CTAs per SM (1..2 in FP64) at the best tile, then re-sort intervals
 * -1 (never), 10, 20, 40 at the best of both, each timed over 80 steps
 * after 40 (the particle order of a new simulation decays over tens of
 * steps, so shorter windows favour no re-sort unduly).  The choice is kept
 * for the class and used by zpic_create for settings left at 0.
 * ms_per_candidate[k] (k < cap, may be NULL) receives each timing in that
 * order (negative: could not run); *n_candidates their number.  Errors as
 * for zpic_autotune. */
int zpic_autotune_all(const zpic_config *cfg, int steps, zpic_tuning *best,
                      double *ms_per_candidate, int cap, int *n_candidates);

/* Tunes the same three settings for a batch of n >= 2 simulations (the
 * batched sweep: many independent simulations advanced by one launch per
 * stage, Sec. 3.2's regions over all of them), by timing the batch itself
 * with each candidate given to every member, in the order of
 * zpic_autotune_all: the tile candidates at `steps` timed steps after 3,
 * then the resident CTAs per SM, then the re-sort intervals over 80 steps
 * after 40.  The full batch is created and destroyed once per candidate
 * (its memory and time are those of the batch).  The choice is kept for
 * this list of configuration classes, and zpic_batch_create with the same
 * list uses it for the settings its members leave at 0; without it those
 * members get 16 x 16 tiles, not the per-class choices of zpic_autotune,
 * which are made for a simulation alone on the GPU.  ms_per_candidate and
 * n_candidates as for zpic_autotune_all.  ZPIC_EINVAL for NULL arguments,
 * n < 2 or steps outside [1, 10000]; ZPIC_ECUDA when no tile candidate
 * ran. */
int zpic_batch_autotune(const zpic_config *cfgs, int n, int steps,
                        zpic_tuning *best, double *ms_per_candidate, int cap,
                        int *n_candidates);

/* Kernel timing: when enabled, zpic_step launches kernels one by one and
 * records a CUDA event pair around each launch on the handle's stream.
 * zpic_profile_read returns, per kernel name, the summed device time (ms)
 * and the number of launches since the last reset (synchronises). */
int zpic_profile_enable(zpic_sim *sim, int enable);
int zpic_profile_read(zpic_sim *sim, char *names, size_t name_len,
                      double *ms_total, int32_t *launches, int cap, int *n,
                      int reset);

/* Batched simulations (independent; same precision): one launch per stage
 * advances all of them over a (simulation, tile) work list, captured in a
 * CUDA graph.  Each member runs the step of Sec. 2.2 exactly as it would
 * alone (bitwise the same in FP32); the work list takes the place of the
 * paper's task scheduler (Sec. 3.2: regions as tasks, over-decomposition
 * of Sec. 4.3), ordered longest first.  zpic_batch_create copies the n
 * configurations (ZPIC_EINVAL if they differ in precision); zpic_batch_step
 * and zpic_batch_sync behave like zpic_step and zpic_sync for all members;
 * zpic_batch_sim gives a view handle for the getters (views are freed with
 * the batch; zpic_destroy on a view is ZPIC_EINVAL).  With n >= 2, members
 * that leave the tile size, re-sort interval or CTAs per SM at 0 take the
 * choice of zpic_batch_autotune for this list of configuration classes if
 * it has run, else a 16 x 16 tile (not the per-class choice of
 * zpic_autotune, made for one simulation alone on the GPU); with n = 1 the
 * rules of zpic_create apply. */
int zpic_batch_create(const zpic_config *cfgs, int n, zpic_batch **out);
int zpic_batch_step(zpic_batch *b, int n);
int zpic_batch_sync(zpic_batch *b);
int zpic_batch_sim(zpic_batch *b, int i, zpic_sim **view);
int zpic_batch_set_stream(zpic_batch *b, void *stream);
int zpic_batch_profile_enable(zpic_batch *b, int enable);
int zpic_batch_destroy(zpic_batch *b);

/* Allocation hooks for the device memory of handles created afterwards
 * (NULL, NULL restores cudaMalloc/cudaFree).  alloc returns a device
 * pointer aligned to 256 bytes or NULL; both get the handle's stream. */
typedef void *(*zpic_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*zpic_free_fn)(void *ptr, size_t bytes, void *stream,
                             void *ctx);
int zpic_set_allocator(zpic_alloc_fn alloc, zpic_free_fn free_fn, void *ctx);

const char *zpic_strerror(int code);
const char *zpic_last_error(void);
int zpic_version(void);

#ifdef __cplusplus
}
#endif
#endif /* ZPIC_H */
