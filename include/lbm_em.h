/*
 * lbm_em.h -- C ABI of the GB300 (sm_103a) lattice Boltzmann Maxwell solver for
 * radiation forces and torques on Janus cylinders (arXiv 2509.22308).
 *
 * Method (paper Sec. III): D3Q7 lattice Boltzmann for TM^z fields (E_z, H_x, H_y),
 *   e_i(r + c_i, t + 1) = 2 e_i^eq(r, t) - e_i(r, t),  h_i likewise   (Eq. LBGK equation)
 *   e_i^eq = (E - c_i x H)/6, h_i^eq = (H + c_i x E)/6 (i != 0), e_0^eq = (eps_r - 1) E
 *                                                       (Eq. equilibrium distribution functions)
 * with a plane-wave source on the left edge, open (first-order extrapolation) edges,
 * PEC cells, Fourier accumulation over one period and the period-averaged Maxwell
 * stress tensor integrated on a closed contour (Sec. II.B, Eq. stress tensor average,
 * Eq. force, Eq. torque), normalised by F0 = pi a E0^2 / 4 and M0 = 2 F0 a.
 *
 * Units: lattice cell = time step = 1, eps0 = mu0 = 1; light travels 1/3 cell per
 * step, so an incident period of T steps has wavelength T/3.  The wave travels
 * along +x; F~x is the drag and F~y the lift towards +y.
 *
 * Conventions shared by every call:
 *  - Arrays of sites are row-major [ny][nx] (x fastest), host memory unless a
 *    name says "device".  The caller owns every buffer it passes; the library
 *    copies what it keeps.
 *  - Every call returns an lbm_em_status; no exception or longjmp crosses the ABI.
 *    lbm_em_last_error() gives a message for the calling thread's last failure.
 *  - Calls on one handle must not overlap (one host thread at a time per handle).
 *  - The library needs a CUDA device; without one (or without the sm_103a
 *    image) create calls fail with LBM_EM_ECUDA.  There is no CPU fallback.
 */
#ifndef LBM_EM_H
#define LBM_EM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBM_EM_OK = 0,
    LBM_EM_EINVAL = 1,     /* bad argument (NULL, size, eps < 1, too many materials ...) */
    LBM_EM_ENOMEM = 2,     /* device or host allocation failed                          */
    LBM_EM_ECUDA = 3,      /* a CUDA runtime call failed (no device, launch error ...)  */
    LBM_EM_EUNSTABLE = 4,  /* a field became non-finite or |E| reached 3 * 2^(20 + k),
                              2^k <= |E0| < 2^(k+1) (sticky)                             */
    LBM_EM_ETIMEOUT = 5,   /* a bounded device-side wait gave up; the handle or batch
                              must then be destroyed (it refuses further steps)         */
    LBM_EM_ESTATE = 6      /* call not valid in the handle's state                       */
} lbm_em_status;

/* Storage of the distributions.  Arithmetic is FP64 for F64, FP32 otherwise;
 * Fourier accumulators and the stress-tensor integral are FP64 in every form. */
typedef enum {
    LBM_EM_F64 = 0,      /* 11 FP64 populations per site (the independent part of the
                            TM^z state; the other five follow from exact invariants)    */
    LBM_EM_F32 = 1,      /* 11 FP32 populations per site                                */
    LBM_EM_F16DEV = 2,   /* FP32 fields (E_z/3, H_x/3, H_y/3) + 11 FP16 scaled
                            deviations f - f^eq per site                                */
    LBM_EM_F32X2 = 3     /* 11 double-float populations per site: pairs of FP32 (hi + lo,
                            ~48 significant bits, FP32 exponent range), FP32-pipe
                            arithmetic by error-free transformations; FP64-class results
                            (the FP64 parity bound holds) at HBM-bound speed on GB300,
                            whose FP64 pipe is 1/64 of its FP32 rate.  Not an IEEE
                            binary64 computation.  One step per launch by default
                            (LBM_EM_FLAG_TWO_STEP selects two); the batch accepts it too */
} lbm_em_precision;

/* Left-edge plane-wave source (Sec. III: the wave enters through the left boundary, the
 * other boundaries let outgoing waves leave).  HARD is the default: energy-stable over
 * hundreds of periods.  OPEN keeps a zero-gradient copy of the scattered part on the left
 * edge as well; with four copy edges a static field can build up around a PEC (a DC
 * line current) and the domain energy grows slowly, without effect on the phasors. */
typedef enum {
    LBM_EM_SRC_HARD = 0,  /* incoming +x populations at x = 0: the exact discrete incident
                             plane wave only (outgoing waves leave freely)               */
    LBM_EM_SRC_OPEN = 1,  /* incoming +x populations at x = 0: zero-gradient copy of the
                             scattered part + the exact discrete incident plane wave     */
    LBM_EM_SRC_NONE = 2   /* no source (all edges open)                                  */
} lbm_em_source_kind;

/* lbm_em_grid.flags: how many time steps one kernel launch advances.  By default FP64 and
 * double-float advance one step per launch; FP32 and FP16-deviation two below 2^20 sites
 * (each tile and its halo are copied to shared memory by the TMA unit and advance two
 * steps there), four from there on (each warp streams a strip of the lattice through four time
 * levels held in registers).  The flags force a mode.  In FP32, FP64 and double-float the
 * result does not depend on the choice: every mode gives the same bits.  In FP16-deviation the
 * four-step mode rounds the stored state to FP16 once per launch instead of once per step, so
 * its bits differ from the other modes by FP16 rounding noise (its runs still give the same
 * bits however they are split, as long as the splits fall on multiples of four steps).
 * Invalid combinations return LBM_EM_EINVAL. */
#define LBM_EM_FLAG_SINGLE_STEP 1  /* always one step per launch                          */
#define LBM_EM_FLAG_TWO_STEP 2     /* two steps per launch for FP32, FP16-dev, double-float */
#define LBM_EM_FLAG_THREE_STEP 8   /* three steps per launch (FP32 only; 28 x 12 tiles)      */
/* four steps per launch (FP32 and FP16-dev): each warp streams a 64-column strip down the
 * lattice and keeps four time levels in registers; FP32 gives the same bits, FP16-dev rounds
 * its stored state once per launch instead of once per step (closer to FP32, other bits) */
#define LBM_EM_FLAG_FOUR_STEP 16
/* TE^z polarization (H_z, E_x, E_y), which the paper leaves for future work (Sec. I): the
 * same scheme and storage (11 planes), incident wave E_y = H_z = E0 sin(w t - k x).  Every
 * call that reports the TM triple (E_z, H_x, H_y) reports (H_z, E_x, E_y) instead: fields,
 * phasors, the stress-tensor contour integral (same form by duality) and the far field (of
 * H_z).  FP64 and FP32 only; LBM_EM_F16DEV with this flag is EINVAL. */
#define LBM_EM_FLAG_TE 4

typedef struct {
    int32_t nx, ny;       /* lattice size, each >= 4                                      */
    int32_t precision;    /* lbm_em_precision                                             */
    int32_t flags;        /* 0 or one of LBM_EM_FLAG_SINGLE_STEP, _TWO_STEP, _THREE_STEP,
                             _FOUR_STEP, optionally | LBM_EM_FLAG_TE                      */
    void *stream;         /* cudaStream_t every kernel of the handle runs on; NULL: the
                             library creates a private non-blocking stream                */
} lbm_em_grid;

typedef struct {
    int32_t period_steps; /* T >= 4: steps per period (wavelength T/3)                    */
    int32_t ramp_steps;   /* >= 0: amplitude ramp sin^2(pi t / (2 ramp)) for t < ramp     */
    int32_t kind;         /* lbm_em_source_kind                                           */
    int32_t reserved;     /* 0                                                            */
    double E0;            /* incident amplitude (the force scale F0 uses it).  The scheme is
                             linear, so the runaway test and the FP16 deviation scale
                             follow it: with 2^k <= |E0| < 2^(k+1) the test fires at
                             |E| >= 3 * 2^(20 + k) and deviations are stored x 2^(10 - k)  */
} lbm_em_source;

/* Janus cylinder (Sec. II): radius a, region II (eps1) where d . n_d > 1e-9 with
 * n_d = (-sin phi0, -cos phi0) and d the offset from the centre, region III (eps2, or
 * PEC) elsewhere inside |d| <= a, vacuum outside.  A homogeneous cylinder is eps1 == eps2. */
typedef struct {
    double a;             /* radius in cells, > 0                                         */
    double phi0;          /* interface orientation, radians                               */
    double eps1;          /* region II relative permittivity, >= 1                        */
    double eps2;          /* region III relative permittivity, >= 1 (ignored if pec2)     */
    int32_t pec2;         /* 1: region III is a perfect electric conductor                */
    int32_t reserved;     /* 0                                                            */
    double cx, cy;        /* centre in lattice coordinates; NaN: ((nx-1)/2, (ny-1)/2)     */
} lbm_em_janus;

/* Stress-tensor contour (Sec. II.B): circle of radius R about (cx, cy), n_points
 * samples phi_k = 2 pi k / n_points, phasors bilinearly interpolated.  The circle
 * must lie strictly inside the lattice (1 <= cx +- R <= nx - 2, same for y). */
typedef struct {
    double cx, cy;        /* centre; NaN: lattice centre                                  */
    double radius;        /* R > 0                                                        */
    int32_t n_points;     /* >= 8, or 0 for 2 ceil(2 pi R)                                 */
    int32_t reserved;     /* 0                                                            */
    double a;             /* cylinder radius used for F0 = pi a E0^2/4, M0 = 2 F0 a       */
} lbm_em_contour;

typedef struct lbm_em lbm_em_t;

/* Create a solver from a host permittivity map eps_map[ny][nx] (each value >= 1) and
 * an optional host PEC mask pec_mask[ny][nx] (non-zero = PEC; NULL = none).  At most
 * 255 distinct permittivities.  Distributions start at zero (time 0).
 * Paper: Sec. III (per-cell eps_r, mu_r = 1), Sec. II (regions I-III). */
lbm_em_status lbm_em_create(const lbm_em_grid *g, const double *eps_map, const uint8_t *pec_mask,
                            const lbm_em_source *s, lbm_em_t **out);

/* Create a solver whose material map is the staircase Janus disc j, rasterised on the
 * device (region ids 0 = vacuum, 1 = region II, 2 = region III).  Sec. II, Sec. IV.A. */
lbm_em_status lbm_em_create_janus(const lbm_em_grid *g, const lbm_em_janus *j,
                                  const lbm_em_source *s, lbm_em_t **out);

/* Return the handle to time 0: distributions, Fourier accumulators and the error flag
 * are cleared on the device (no allocation).  Asynchronous on the handle's stream. */
lbm_em_status lbm_em_reset(lbm_em_t *h);

/* Re-rasterise a Janus disc j into the handle's material map in place (same lattice;
 * region ids 0/1/2 as in lbm_em_create_janus), e.g. the next cell of a design map.
 * Does not touch the distributions (call lbm_em_reset for a fresh run).  Asynchronous
 * on the handle's stream.  Sec. II. */
lbm_em_status lbm_em_set_janus(lbm_em_t *h, const lbm_em_janus *j);

/* Release every resource of the handle (NULL is accepted). */
lbm_em_status lbm_em_destroy(lbm_em_t *h);

/* Enqueue n >= 0 time steps (fused stream-collide over every site, source, open
 * edges, PEC), Eq. (LBGK equation).  Asynchronous on the handle's stream. */
lbm_em_status lbm_em_step(lbm_em_t *h, int64_t n);

/* Wait for the handle's stream; returns LBM_EM_EUNSTABLE if any step flagged a
 * non-finite or runaway field since creation (the flag is sticky), LBM_EM_ETIMEOUT if a
 * tile copy of a step never completed.  After LBM_EM_ETIMEOUT a copy may still have been in
 * flight when its thread block left, so the handle's state is undefined: lbm_em_step and
 * lbm_em_accumulate then return LBM_EM_ESTATE, and the handle must be destroyed. */
lbm_em_status lbm_em_sync(lbm_em_t *h);

/* Time steps one launch of the handle's step kernel advances (1, 2, 3 or 4), the mode that
 * lbm_em_grid.flags forced or the default chose for the form and lattice size.  Runs of fewer
 * steps, and the steps that bring an odd start time to an even one for two-step launches,
 * take single-step launches. */
lbm_em_status lbm_em_get_steps_per_launch(lbm_em_t *h, int32_t *n);

/* Current time step count (host view; equals the number of steps enqueued). */
lbm_em_status lbm_em_get_time(lbm_em_t *h, int64_t *t);

/* Define the stress-tensor contour and clear the Fourier accumulators (Sec. III:
 * phasors from Fourier analysis over one period). */
lbm_em_status lbm_em_set_contour(lbm_em_t *h, const lbm_em_contour *c);

/* Enqueue n steps that also add (E_z, H_x, H_y)(t) * e^{i w t}, w = 2 pi / T, at every
 * site the contour interpolates from, before each step's collision.  Requires a contour. */
lbm_em_status lbm_em_accumulate(lbm_em_t *h, int64_t n);

/* From the accumulators (n accumulated steps, phasor = (2/n) * sum): the
 * period-averaged stress tensor on the contour -> out[3] = {F~x, F~y, M~z}
 * (Eq. stress tensor average, force, torque; F0, M0 of Sec. II.B).  Synchronous. */
lbm_em_status lbm_em_contour_integral(lbm_em_t *h, double out[3]);

/* set_contour(c) + accumulate(T) + contour_integral(out): advances one period. */
lbm_em_status lbm_em_force_torque(lbm_em_t *h, const lbm_em_contour *c, double out[3]);

/* As lbm_em_contour_integral, but asynchronous: the three doubles are written to the
 * device buffer d_out (8-byte aligned, caller-owned) on the handle's stream. */
lbm_em_status lbm_em_contour_integral_device(lbm_em_t *h, double *d_out);

/* As lbm_em_force_torque, but asynchronous with the result in the device buffer d_out:
 * several handles on different streams can then run their periods concurrently.
 * (Setting a contour that differs from the current one allocates and synchronises.) */
lbm_em_status lbm_em_force_torque_device(lbm_em_t *h, const lbm_em_contour *c, double *d_out);

/* Far-field scattering intensity |S(phi)|^2 = k0 r |E^S|^2 / |E^I|^2 (Sec. II.A, Eq.
 * scattering intensity) at n_angles observation angles (radians, lattice frame: 0 is
 * forward, along +x) from the accumulated phasors on the current contour, by a
 * near-to-far-field transform (Green's theorem with the Hankel asymptote; the scattered
 * near field is the phasor minus the lattice's exact incident plane wave).  Uses the
 * lattice wavenumber of the source period.  Host arrays; synchronous. */
lbm_em_status lbm_em_far_field(lbm_em_t *h, const double *angles, int32_t n_angles, double *s2);

/* Total electromagnetic energy of the lattice at the current time,
 * W = sum over sites of (eps_r E_z^2 + H_x^2 + H_y^2) / 2 (lattice units), the quantity whose
 * approach to a constant the paper uses as its convergence criterion (Sec. III).  Synchronous. */
lbm_em_status lbm_em_energy(lbm_em_t *h, double *W);

/* Run whole periods until the energy sampled at the end of each period (so always at
 * the same phase) has changed by at most tol * W twice in a row, after at least
 * min_periods - 1 periods, or until max_periods - 1 periods have run; then (one step
 * later if it converged, as the batched path does) one accumulated period and the
 * contour integral into out[3] as lbm_em_force_torque.  *steps_run (may be NULL)
 * receives the number of steps taken.  Convergence criterion of Sec. III. */
lbm_em_status lbm_em_run_converged(lbm_em_t *h, const lbm_em_contour *c, double tol, int32_t min_periods,
                                   int32_t max_periods, double out[3], int64_t *steps_run);

/* Fields at the current time into host arrays [ny][nx] (any may be NULL).  Synchronous. */
lbm_em_status lbm_em_get_fields(lbm_em_t *h, double *ez, double *hx, double *hy);

/* Phasors at the contour's stencil sites: site_xy[2*k] = x, [2*k+1] = y and
 * phasors[6*k .. 6*k+5] = Re/Im of E_z, H_x, H_y (already scaled by 2/n).  With
 * NULL arrays only *n_sites is written.  Synchronous. */
lbm_em_status lbm_em_get_phasors(lbm_em_t *h, int32_t *site_xy, double *phasors, int32_t *n_sites);

/* Material ids [ny][nx] (host) and, if eps_table is not NULL, eps_table[256] with the
 * relative permittivity of each id (0 for PEC ids, 1 for unused ids).  Synchronous. */
lbm_em_status lbm_em_get_material(lbm_em_t *h, uint8_t *ids, double *eps_table);

/* Checkpoint: with buf == NULL writes the size needed to *bytes; otherwise copies the
 * distributions, time and accumulators into buf (capacity *bytes).  Synchronous. */
lbm_em_status lbm_em_save_state(lbm_em_t *h, void *buf, size_t *bytes);

/* Restore a checkpoint written by lbm_em_save_state of a handle with the same grid,
 * precision, source and contour.  A resumed run equals an unsplit run bit for bit. */
lbm_em_status lbm_em_load_state(lbm_em_t *h, const void *buf, size_t bytes);

/* Message of the calling thread's last failed call ("" if none). */
const char *lbm_em_last_error(void);

/* Diagnostic of the device-side bounded waits (the paper has no counterpart).  The
 * TMA-staged kernels wait on an mbarrier for their tile copies and give up after a limit
 * (about 2e9 clock cycles), reporting LBM_EM_ETIMEOUT instead of spinning forever.  This
 * call runs the same wait in one block on an mbarrier that nothing arrives on, for at most
 * limit_cycles (1 .. 2e9) clock cycles, and reports it the way a kernel's timeout is
 * reported: LBM_EM_ETIMEOUT is the expected result; the device stays usable.  Synchronous,
 * on the legacy default stream; LBM_EM_EINVAL for a limit outside the range. */
lbm_em_status lbm_em_probe_bounded_wait(int64_t limit_cycles);

/* Diagnostic of the FP64 pipe (the paper has no counterpart), the ceiling of the FP64 step on
 * GB300: enqueues on `stream` (a cudaStream_t; NULL: the legacy default stream) one launch of
 * 8 independent FP64 fused multiply-add chains of `iters` steps (>= 1) in each of 8 x 256
 * threads per SM, and writes the number of FMAs the launch performs to *fma_per_launch.  Time
 * it with events on the same stream: FMAs / time is the measured FP64 operation rate.
 * Asynchronous; LBM_EM_EINVAL for iters < 1 or a NULL output. */
lbm_em_status lbm_em_probe_fp64_fma(void *stream, int64_t iters, double *fma_per_launch);

/* Check of the FP16-deviation rebuild that the four-step kernel uses (the paper has no
 * counterpart): f = eq2 / 2 - g 2^m with each FP16 deviation g taken straight into a
 * mixed-precision FMA, against converting g to FP32 first and using the FP32 FMA.  g2[n] holds
 * pairs of FP16 deviations (low and high half, both are used), eq2[n] FP32 values of 2 f^eq, m
 * the exponent of the inverse scale (-24 .. 15: -2^m is an FP16 number); host arrays, read
 * only.  *mismatches = the number of the 2 n results whose bits differ (a NaN against a NaN
 * counts as equal).  Synchronous, on the legacy default stream; LBM_EM_EINVAL for n < 1, m out
 * of range or a NULL pointer, LBM_EM_ENOMEM if the device copies cannot be allocated. */
lbm_em_status lbm_em_probe_f16_rebuild(const uint32_t *g2, const float *eq2, int64_t n, int32_t m,
                                       int64_t *mismatches);

/* Bytes this library has copied host -> device (*h2d) and device -> host (*d2h) in the calls
 * of the solver and the batch since it was loaded (either pointer may be NULL): e.g. the
 * transfer volume of one end-to-end run is the difference of two readings.  The library
 * counts each copy when it enqueues it. */
lbm_em_status lbm_em_transfer_bytes(uint64_t *h2d, uint64_t *d2h);

/* Host-side fault injection for tests of the clean-up paths (the paper has no counterpart).
 * Every device and pinned-host allocation the library makes counts as one attempt.  With
 * fail_at > 0 the fail_at-th attempt after this call fails as if the device or host were out
 * of memory, so the call that made it returns LBM_EM_ENOMEM after releasing what it had
 * already allocated; fail_at = 0 disarms the hook.  *live (may be NULL) receives the number
 * of device buffers and pinned blocks that handles and batches hold at the time of the call
 * (pinned blocks parked for reuse between handles are not held by any).  Process-wide and
 * thread-safe; nothing is injected on the device.  LBM_EM_EINVAL for fail_at < 0. */
lbm_em_status lbm_em_test_alloc_hook(int64_t fail_at, int64_t *live);

/* Rasterise a Janus disc on the device into host region ids [ny][nx]
 * (0 vacuum, 1 region II, 2 region III).  Sec. II, Sec. IV.A staircase. */
lbm_em_status lbm_em_rasterize_janus(const lbm_em_janus *j, int32_t nx, int32_t ny, uint8_t *regions);

/* Size of the fixed device array used by lbm_em_rasterize_janus_noalloc. */
#define LBM_EM_NOALLOC_RASTER_BYTES (4u * 1024u * 1024u)

/* The same rasterisation as lbm_em_rasterize_janus, for callers that must not allocate
 * device memory: for example an application whose own memory pool already holds the
 * device's free memory, or a latency-critical loop in which cudaMalloc / cudaFree would
 * synchronise the device.  The paper has no counterpart; this is a service of the library.
 * It calls no cudaMalloc, cudaFree or other allocating routine: the region ids are written
 * into one 4 MiB array compiled into this library's device image (every GPU that loads the
 * library holds it until the process exits) and then copied into regions[ny][nx] (host).
 *  - ny * (nx rounded up to a multiple of 32) must not exceed LBM_EM_NOALLOC_RASTER_BYTES;
 *    a larger request returns LBM_EM_EINVAL with a message and launches nothing.
 *  - Each call looks up the array's address in the current context (cudaGetSymbolAddress,
 *    which allocates nothing), so the address stays right after the caller resets the
 *    device or recreates its primary context.
 *  - Runs on the legacy default stream and copies synchronously, returning once regions is
 *    filled.  Neither is allowed while a global- or thread-local-mode stream capture is
 *    active, so no call may overlap one; such a call returns LBM_EM_ECUDA.
 *  - Every call shares the one array, which keeps the last call's contents; calls that
 *    overlap on the GPU (several host threads at once) race, so serialise them. */
lbm_em_status lbm_em_rasterize_janus_noalloc(const lbm_em_janus *j, int32_t nx, int32_t ny, uint8_t *regions);

/* ---- batched design diagrams (Sec. IV maps over eps and phi0) ---------------------- */

typedef struct {
    int32_t nx, ny;          /* lattice of this instance                                   */
    int32_t period_steps;    /* T                                                          */
    int32_t periods;         /* run length in periods; the last one is Fourier-averaged    */
    int32_t ramp_steps;      /* source ramp                                                */
    int32_t n_points;        /* contour samples (0: 2 ceil(2 pi R))                         */
    double E0;               /* incident amplitude                                         */
    double contour_radius;   /* R                                                          */
    lbm_em_janus janus;      /* geometry (centre NaN: lattice centre)                      */
} lbm_em_instance;

typedef struct {
    int32_t precision;       /* LBM_EM_F32, LBM_EM_F64 or LBM_EM_F32X2                      */
    int32_t tile_w, tile_h;  /* tile shape (tile_w 32/40/64/128/256, tile_h <= 16); 0: autotuned.
                                64 x 8, 32 x 16 and 40 x 12 with 3 CTAs per SM are the
                                configurations of the two-steps-per-launch kernel (FP32,
                                conv_tol 0: each tile and its halo are copied to shared memory
                                by the TMA unit and advance two steps there, same bits; 40 is
                                valid for it only).  With nothing pinned the autotuner times
                                those three when they apply, else the one-step shapes      */
    int32_t ctas_per_sm;     /* persistent CTAs per SM; 0: autotuned.  With
                                steps_per_launch 4: 1 .. 3 runs the four-step kernel on a
                                persistent grid of that many blocks per SM whose warps take
                                the work units in turn (0: one warp per unit, the default) */
    int32_t min_periods;     /* convergence exits: fewest periods an instance runs         */
    int32_t source_kind;     /* lbm_em_source_kind of every instance (0: HARD)              */
    double conv_tol;         /* 0: every instance runs its `periods`; > 0: an instance stops
                                early once its domain energy, sampled at each period end,
                                changes by <= conv_tol * W twice in a row (Sec. III), then
                                runs one accumulated period; `periods` is the maximum     */
    void *stream;            /* cudaStream_t; NULL: private stream                         */
    int32_t polarization;    /* 0: TM^z (E_z, H_x, H_y), the paper's case; 1: TE^z (H_z,
                                E_x, E_y) for every instance (see LBM_EM_FLAG_TE)          */
    int32_t steps_per_launch;/* 0: autotuned; 1, 2 or 4 pins the steps one launch advances.
                                4 (FP32, conv_tol 0, nothing else pinned): one warp per work
                                unit streams a strip of 56 columns and a row segment of an
                                instance through four time levels held in registers (the
                                autotuner picks the segment height, 64, 128 or 256 rows); same
                                bits as one step per launch.  2: the TMA tile kernel above.  With 0 the
                                autotuner times every kind that applies                    */
} lbm_em_batch_opts;

typedef struct lbm_em_batch lbm_em_batch_t;

/* Pack n instances (uneven sizes allowed) into one multi-domain layout on the device: a
 * design map of Sec. IV (one instance per parameter cell, each the single-domain problem of
 * Sec. II-III).  specs[0..n) and *o are copied (the caller keeps them); *out receives a handle
 * the library owns until lbm_em_batch_destroy.  Instances sharing a lattice size, contour and
 * period share one contour description and phase table.  Synchronous: with a tile shape or
 * CTA count not pinned, the autotuner times a few steps of each candidate on the packed data
 * and clears the state.  Errors: LBM_EM_EINVAL for a bad option or instance (the message
 * names it), LBM_EM_ENOMEM / LBM_EM_ECUDA on device failure or without a GPU. */
lbm_em_status lbm_em_batch_create(const lbm_em_instance *specs, int32_t n,
                                  const lbm_em_batch_opts *o, lbm_em_batch_t **out);

/* Rasterise every instance (Sec. II), run each for its periods (Eq. LBGK equation, the last
 * period with the Fourier accumulation of Sec. III) in kernels over the packed tiles or work
 * units replayed under a CUDA graph, then the contour integral of each (Sec. II.B).  A
 * second call starts again from rest.  Asynchronous on the batch's stream; returns launch
 * errors only: per-instance failures come back through lbm_em_batch_results. */
lbm_em_status lbm_em_batch_run(lbm_em_batch_t *b);

/* Wait for the run and fetch: out[3*i .. 3*i+2] = {F~x, F~y, M~z} of instance i (normalised
 * by F0, M0 of Sec. II.B) and status[i] per instance (LBM_EM_OK, LBM_EM_EUNSTABLE for a
 * runaway field, LBM_EM_ETIMEOUT for a tile copy that never completed); caller-owned host
 * arrays of 3 n doubles and n int32, either may be NULL.  Returns LBM_EM_ETIMEOUT or
 * LBM_EM_EUNSTABLE if any instance has that status, LBM_EM_ESTATE before the first run.
 * After LBM_EM_ETIMEOUT lbm_em_batch_run returns LBM_EM_ESTATE: destroy the batch. */
lbm_em_status lbm_em_batch_results(lbm_em_batch_t *b, double *out, int32_t *status);

/* Steps each instance ran in the last lbm_em_batch_run (its run length, shortened by a
 * convergence exit when conv_tol > 0), steps[n].  Synchronous. */
lbm_em_status lbm_em_batch_steps(lbm_em_batch_t *b, int64_t *steps);

/* Chosen tile shape and CTAs per SM (after autotuning), for reporting.  With four steps per
 * launch: 56 (the strip width), the row-segment height and the kernel's resident blocks per
 * SM. */
lbm_em_status lbm_em_batch_config(lbm_em_batch_t *b, int32_t *tile_w, int32_t *tile_h,
                                  int32_t *ctas_per_sm);

/* Steps one launch of the batch's chosen kernel advances (1, 2 or 4). */
lbm_em_status lbm_em_batch_steps_per_launch(lbm_em_batch_t *b, int32_t *n);

/* Release every resource of the batch (NULL is accepted): waits for the work queued on the
 * batch's stream, frees its device memory and graphs, and destroys the stream if the library
 * created it.  Always LBM_EM_OK for a batch from lbm_em_batch_create or NULL. */
lbm_em_status lbm_em_batch_destroy(lbm_em_batch_t *b);

#ifdef __cplusplus
}
#endif
#endif /* LBM_EM_H */
