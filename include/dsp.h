/*
 * dsp.h -- C ABI of the GB300 split-operator solver for pair production in
 * graphene (massless Dirac equation in momentum space, arXiv 1607.03062).
 *
 * Units: hbar = v_F = e = 1; momenta and energies in eV, time in hbar/eV.
 *
 * What the library computes (the paper's method, Sec. II and III):
 *   every grid momentum p carries an independent two-component spinor psi(p).
 *   It starts as the negative-energy free spinor v(p + A_in) (Sec. II, Eq.
 *   (free_spin1..4), normalised to 1) and is stepped N times by the midpoint
 *   exponential of Sec. III, Eq. (approx_time) in its closed form
 *       U_n = I cos(dt |P_n|) - i (valley sigma.P_n / |P_n|) sin(dt |P_n|),
 *       P_n = p + A(t_i + (n + 1/2) dt).
 *   The result is projected on the positive-energy spinor u(p + A_out),
 *   |c+(p)|^2 = |u^dag psi(t_f)|^2, and reduced to the pair density of Sec. II
 *   Eq. (pair_prod_homo) with degeneracy 4 (spin x valley):
 *       n = 4/(2 pi)^2 * hx * hy * sum_p |c+(p)|^2        [eV^2].
 *
 * Grid: nx by ny cell-centred nodes, p_x(i) = px_min + (i + 1/2)(px_max - px_min)/nx,
 * same for y; arrays are row-major [ny][nx] with x fastest.
 *
 * Conventions for every entry point:
 *   - returns a dsp_status and never aborts or traps; inputs are validated
 *     before anything is launched;
 *   - host arrays passed in are copied before the call returns and never kept;
 *   - device pointers passed in are owned by the caller and must stay valid
 *     until the work queued on the grid's stream has finished;
 *   - work is queued on the grid's CUDA stream (the stream given at creation;
 *     NULL means the legacy default stream); only dsp_reduce_density, dsp_solve,
 *     dsp_solve_host and the server's step synchronise with the host;
 *   - a CUDA error is latched in the handle: that call and every later call on
 *     the handle return DSP_E_CUDA (destroy still frees what it can);
 *   - handles are not thread safe: one host thread per handle at a time
 *     (distinct handles may be used from different host threads).
 */
#ifndef DSP_H
#define DSP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t dsp_status;
#define DSP_OK 0
#define DSP_E_INVALID (-1) /* a bad argument (NaN, size, enum, NULL ...)          */
#define DSP_E_NOMEM (-2)   /* device or host allocation failed, or over budget    */
#define DSP_E_CUDA (-3)    /* a CUDA call failed (latched in the handle)          */
#define DSP_E_STATE (-4)   /* call out of order (no pulse, steps past the end ...) */
#define DSP_E_CFL (-5)     /* dt * max|p + A| > pi: the step condition of Sec. III */
#define DSP_E_TIMEOUT (-6) /* a bounded device-side wait gave up (error flag set) */
#define DSP_E_BOUNDS (-7)  /* an out-of-range device index, found only by a library
                              built with -DDSP_BOUNDS_CHECK (accesses are skipped) */

/* Arithmetic of the evolution. */
#define DSP_FP64 0       /* the spinor and its update in FP64; in the EXACT scheme the
                            small parts cos(theta) - 1 and sin(theta)/theta - 1 are
                            evaluated in double-float FP32 arithmetic (~1e-19
                            absolute, below an FP64 ulp of the state)               */
#define DSP_FP32_MIXED 1 /* spinor in compensated FP32 (hi + lo); dt P_n formed as
                            dt p_hi + (dt A_n + dt p_lo) with dt p an FP32 hi/lo
                            pair and dt A_n one FP32 per step, rounded on the host
                            with error feedback; the trigonometric factors of
                            the phase argument dt|P| (cos/sin series, or the tan
                            series of step groups) in FP32; initial state in FP64 */

/* Time-step scheme. */
#define DSP_SCHEME_EXACT 0     /* the paper's closed-form exponential (Sec. III)    */
#define DSP_SCHEME_STRANG_XY 1 /* e^{-i dt Px sx/2} e^{-i dt Py sy} e^{-i dt Px sx/2},
                                  a sigma_x / sigma_y split (not in the paper)      */
#define DSP_SCHEME_MAGNUS4 2   /* fourth-order Magnus with two Gauss points per step,
                                  exp(dt/2 (A1 + A2) - sqrt(3) dt^2/12 [A1, A2]),
                                  A_k = -i valley sigma.P(t_n + (1/2 -/+ sqrt(3)/6) dt):
                                  the higher-order decomposition Sec. III mentions.
                                  Its pulse tables hold TWO samples per step (the
                                  Gauss points): [n_steps][2][2]                    */

typedef struct dsp_grid dsp_grid;

/* Bytes of device state one grid needs: 32 bytes per point for both
 * precisions (FP64: two complex doubles; FP32_MIXED: hi and lo float4 planes).
 * Returns -1 on invalid sizes or precision.  (Memory layout of this library:
 * the paper has no counterpart.) */
int64_t dsp_state_bytes(int32_t nx, int32_t ny, int32_t precision);

/* Creates a grid.  nx, ny >= 1 and nx*ny <= 2^31 - 1; px_min < px_max and
 * py_min < py_max, all finite; precision DSP_FP64 or DSP_FP32_MIXED; scheme
 * DSP_SCHEME_*; valley +1 (K+) or -1 (K-, H = -sigma.P, Sec. II Eq.
 * (dirac_eq_mom)).  cuda_stream is a cudaStream_t (NULL: legacy stream).
 * state_dev: NULL lets the library allocate the spinor state; otherwise a
 * caller-owned device buffer of at least dsp_state_bytes() bytes, 16-byte
 * aligned, kept alive until dsp_destroy_grid.  On success *out is the handle.
 * Defined by Sec. II (grid of independent momenta, Eq. (pair_prod_homo)). */
dsp_status dsp_create_grid(int32_t nx, int32_t ny, double px_min, double px_max, double py_min,
                           double py_max, int32_t precision, int32_t scheme, int32_t valley,
                           void *cuda_stream, void *state_dev, int64_t state_dev_bytes,
                           dsp_grid **out);

/* Creates a grid that holds the rows [row_begin, row_end) of the nx by ny grid
 * on the box (0 <= row_begin < row_end <= ny): a band for sharding one grid's
 * momenta across devices (they are independent, Sec. III).  Its nodes are the
 * full grid's, p_y(j) = py_min + (j + 1/2)(py_max - py_min)/ny for the global
 * row j, and every choice that depends on the grid (the step condition, the
 * series degrees, the step-group size: all taken over the full box) is the full
 * grid's, so each point of the band evolves and projects bitwise as in the
 * full grid.  Arrays (state, map) hold the band's rows only,
 * [row_end - row_begin][nx]; dsp_state_bytes(nx, row_end - row_begin, ...)
 * sizes the state.  dsp_reduce_density returns the band's share of the full
 * grid's density (the same 4/(2 pi)^2 hx hy factor, summed over the band's
 * points): the shares of all bands add up to the full density up to rounding
 * (their partial sums are grouped differently).  Other arguments and errors as
 * in dsp_create_grid; nx * (row_end - row_begin) <= 2^31 - 1. */
dsp_status dsp_create_band(int32_t nx, int32_t ny, int32_t row_begin, int32_t row_end,
                           double px_min, double px_max, double py_min, double py_max,
                           int32_t precision, int32_t scheme, int32_t valley, void *cuda_stream,
                           void *state_dev, int64_t state_dev_bytes, dsp_grid **out);

/* keep = 1 (the default): every launch leaves the spinor state in device
 * memory.  keep = 0: the launch that takes the last step and projects in the
 * same kernel (dsp_solve, dsp_solve_host) does not write the final state back,
 * saving 32 bytes of HBM writes per point when only the map and the density
 * are wanted.  The final state is then gone: dsp_project, dsp_solve and
 * dsp_save_state return DSP_E_STATE until the next dsp_set_pulse or
 * dsp_load_state.  The map and the density are bitwise the same either way.
 * Not in the paper (a memory-traffic option). */
dsp_status dsp_set_keep_final_state(dsp_grid *g, int32_t keep);

/* Sets the pulse: a_mid is a host array [n_steps][2] of (A_x, A_y) sampled at
 * the step midpoints t_i + (n + 1/2) dt (Sec. III, Eq. (approx_time)) -- for
 * DSP_SCHEME_MAGNUS4 it is [n_steps][2][2], (A_x, A_y) at t_i + (n + 1/2 -
 * sqrt(3)/6) dt then at t_i + (n + 1/2 + sqrt(3)/6) dt (dsp_sample_pulse_gauss
 * fills it); the same holds for dsp_solve_host and dsp_server_submit; a_in and
 * a_out are the asymptotic potentials A^in, A^out of Sec. II (host, 2 doubles
 * each).  All values finite, dt > 0 (dt >= 0 when n_steps == 0), n_steps >= 0.
 * Copies and converts the table to the device, resets the state to
 * v(p + A_in) and the step cursor to 0.  Returns DSP_E_CFL when
 * dt * max_{n, p in box} |p + A_n| > pi (the step condition of Sec. III).
 * Not ordered against work already queued that still reads the old table:
 * the library orders it on the grid's stream. */
dsp_status dsp_set_pulse(dsp_grid *g, const double *a_mid, int64_t n_steps, double dt,
                         const double a_in[2], const double a_out[2]);

/* Advances every point by `steps` time steps (Sec. III, Eq. (ev_op_dt)) from
 * the cursor; steps >= 0 and cursor + steps <= n_steps, else DSP_E_STATE.
 * The spinors stay on the device.  Evolving in pieces gives bitwise the same
 * state as evolving at once when every piece ends on a multiple of 16 steps:
 * with grouped steps (group_steps G > 1 in dsp_get_info) the steps
 * (G j, ..., G j + G - 1) are multiplied into one operator before the
 * compensated update, and a piece boundary inside such a group changes
 * rounding only.  With G = 1 any split is bitwise invariant.  Asynchronous. */
dsp_status dsp_evolve(dsp_grid *g, int64_t steps);

/* Projects psi(t_f) on u(p + A_out) (Sec. II, Eq. (pair_prod_homo)) and writes
 * the |c+|^2 map, [ny][nx] row-major, to the caller's device buffer map_dev:
 * double for DSP_FP64, float for DSP_FP32_MIXED.  Needs cursor == n_steps
 * (DSP_E_STATE otherwise).  Also leaves per-tile FP64 partial sums for
 * dsp_reduce_density.  Points with |p + A_out| == 0 get |c+|^2 = 0.
 * DSP_FP64 evaluates |c+|^2 in double-float arithmetic (pairs of FP32, about
 * 48 bits, ~1e-14 absolute); DSP_FP32_MIXED in FP32 from the hi parts of the
 * state (error below ~4e-7 |c+|, the size of the float map's own rounding).
 * Either way it is the same code as the projection fused into the last evolve
 * launch, so the two give the same bits.  A projection of
 * a state already on the device reads it (32 bytes per point) without writing
 * it back and writes the map (4 or 8 bytes per point).  Asynchronous. */
dsp_status dsp_project(dsp_grid *g, void *map_dev);

/* Reduces the last projection to the pair density n (eV^2) in a fixed order
 * (deterministic: bitwise the same on every run; double-float pairwise trees
 * over granules of 256 consecutive points, then an FP64 sum of the granules),
 * times
 * 4/(2 pi)^2 * hx * hy (Sec. II, Eq. (pair_prod_homo), degeneracy 4).  Needs a
 * projection since the last dsp_set_pulse (DSP_E_STATE otherwise).  Writes
 * *n_host; synchronises the grid's stream. */
dsp_status dsp_reduce_density(dsp_grid *g, double *n_host);

/* Pair density of a |c+|^2 map that ALLOCATES NOTHING.  The paper has no
 * counterpart: this exists for callers that cannot call cudaMalloc -- a host
 * application or framework that already owns the device memory through its
 * own allocator, or a latency-critical loop where cudaMalloc/cudaFree (which
 * can synchronise the device) are not allowed.
 *   map_dev: the caller's device map, nx*ny values row-major [ny][nx], double
 *     for DSP_FP64 or float for DSP_FP32_MIXED (as written by dsp_project);
 *   the box and nx, ny give hx = (px_max - px_min)/nx, hy likewise, and
 *   *n_host receives 4/(2 pi)^2 * hx * hy * sum |c+|^2, the quantity
 *   dsp_reduce_density returns, summed in the same fixed order (bitwise equal
 *   to it for an FP64 map).
 * Scratch: a static device array inside the library sized for at most
 * DSP_NOALLOC_MAX_POINTS points (one double per 256 points, about 2 MB, held
 * on every GPU that loads the library until the process exits); larger maps are refused with
 * DSP_E_INVALID before anything is queued.  The first call made with a given
 * device current looks up the array's device address (cudaGetSymbolAddress)
 * and caches it for the rest of the process; make that first call before any
 * stream capture.  A cudaDeviceReset of that device after the first call is
 * not supported (the cached address would be stale).  Every call overwrites
 * the whole scratch it reads, so no state leaks between calls, but all calls
 * share the one array: calls that overlap on the GPU (other streams, other
 * host threads) race and must be serialised by the caller.  Work is queued on
 * cuda_stream (NULL: legacy stream), which the call synchronises.  Errors left
 * by earlier launches of the caller's are cleared first, so DSP_E_CUDA
 * reports this call's own. */
#define DSP_NOALLOC_MAX_POINTS 67108864
dsp_status dsp_density_noalloc(const void *map_dev, int32_t precision, int32_t nx, int32_t ny,
                               double px_min, double px_max, double py_min, double py_max,
                               void *cuda_stream, double *n_host);

/* The whole hot path in one call: evolves the remaining steps (Sec. III, Eq.
 * (ev_op_dt)) with the projection fused into the same kernel, writes map_dev
 * (may be NULL: then an internal map is used) and the density (Sec. II, Eq.
 * (pair_prod_homo)) to *n_host (may be NULL).  Synchronises when n_host is
 * not NULL. */
dsp_status dsp_solve(dsp_grid *g, void *map_dev, double *n_host);

/* The whole hot path with the time axis split into `segments` pieces that run
 * in parallel (for grids too small to fill the GPU).  The evolution operator
 * is the time-ordered product of the step operators (Sec. III, Eq. (ev_op_dt));
 * the product is associative, so each segment's product is formed on its own
 * (as its first column: every step operator is SU(2), [[a, -conj(b)], [b,
 * conj(a)]], so the column (a, b) determines it), then the segments are
 * multiplied onto v(p + A_in) in time order in FP64.  Same steps, same results
 * as dsp_solve up to rounding (not bitwise).  segments = 0 picks enough for one
 * segment-tile per SM in FP64, one per two SMs in FP32_MIXED (at least 16
 * steps per segment); needs cursor == 0
 * (DSP_E_STATE otherwise).  Scratch: segments * 32 bytes per point, allocated
 * by the library (at most 16 GB, else DSP_E_INVALID).  map_dev and n_host as
 * in dsp_solve. */
dsp_status dsp_solve_segmented(dsp_grid *g, int32_t segments, void *map_dev, double *n_host);

/* End to end with host buffers: copies the host pulse table in (as
 * dsp_set_pulse), runs dsp_solve (Sec. III and Sec. II, as there), and copies
 * the |c+|^2 map (double or float by precision, nx*ny values) back to map_host
 * (may be NULL) and the density to *n_host.  Synchronises. */
dsp_status dsp_solve_host(dsp_grid *g, const double *a_mid, int64_t n_steps, double dt,
                          const double a_in[2], const double a_out[2], void *map_host,
                          double *n_host);

/* Advances several grids, each by steps[i] (same rules as dsp_evolve), in one
 * batched launch per precision present (a launch carries at most 96 grids;
 * more are split over further launches).  The momenta of all the grids are
 * independent (Sec. III: every p carries its own spinor), so the batch only
 * shares launches.  All grids must share one CUDA stream; work goes on that
 * stream.  Results are bitwise identical to advancing each grid alone.  Each
 * grid keeps its own device error word: a bounded wait that runs out (or a
 * bounds-check hit) in one grid's tiles is reported, and latched, by that
 * grid's next synchronising call, not by the others'. */
dsp_status dsp_evolve_batch(dsp_grid *const *grids, const int64_t *steps, int32_t count);

/* Cursor and pulse length of a grid (bookkeeping: the paper has no
 * counterpart). */
dsp_status dsp_get_cursor(const dsp_grid *g, int64_t *cursor, int64_t *n_steps);

/* What the library chose for the current pulse: the degrees (in theta^2) of
 * the cos(theta) and sin(theta)/theta series used per step (picked so their
 * truncation error over all n_steps stays below 1e-6 in FP32_MIXED, 1e-16 in
 * FP64), theta_max = dt * max|p + A_n| over the box, the tile count, and
 * group_steps G: the number of step operators multiplied into one before each
 * compensated update (FP32_MIXED, every scheme: the largest of 16, 8, 4, 2 with
 * G * theta_max <= 0.27 for EXACT and STRANG_XY, <= 0.2 for MAGNUS4, else 1; 1
 * in FP64), and tan_degree, the degree in theta^2 of the groups' tan series
 * (EXACT: tan(theta)/theta; STRANG_XY: tan and sec; MAGNUS4: tan|n|/|n| in
 * |n|^2; 0 when G = 1).  Not in the paper: with G > 1 the update is paid once
 * per group.  The groups multiply the steps divided by the cosine on their
 * diagonal (EXACT and STRANG_XY: the real diagonal cos(theta), so a step of
 * the product costs 8 multiply-adds instead of 12; MAGNUS4: cos|n|) and divide
 * the product by the square root of its determinant, so the applied operator
 * is unitary to FP32 rounding. */
typedef struct {
    int32_t nx, ny, precision, scheme, valley;
    int32_t cos_degree, sinc_degree;
    int32_t n_tiles;
    int64_t n_steps, cursor;
    double dt, theta_max;
    int32_t group_steps;
    int32_t row_begin;  /* first global row (0 unless the grid is a band)      */
    int32_t ny_total;   /* rows of the full grid (ny unless the grid is a band) */
    int32_t row_strips; /* 1: evolve launches tile the grid in row strips of 4 rows
                           x 256 columns (nx a multiple of 256; FP32_MIXED every
                           scheme, FP64 EXACT and STRANG_XY), sharing each step's
                           momentum work across a strip; 0: contiguous tiles of
                           1024 points.  n_tiles counts the tiles of the tiling
                           in use. */
    int32_t tan_degree; /* see above */
} dsp_grid_info;
/* Fills *info for the grid's current pulse (the fields above; bookkeeping,
 * the paper has no counterpart). */
dsp_status dsp_get_info(const dsp_grid *g, dsp_grid_info *info);

/* Test hook for the failure path (not in the paper).  The next launch on this
 * grid announces its first A(t) chunk to the CTA's mbarrier but never copies
 * it, so every CTA's bounded wait for it runs out (after about 2 s).  The CTA
 * then sets the launch's error word and returns: nothing faults, traps or
 * hangs, and the CUDA context stays usable.  The next synchronising call on
 * the grid returns DSP_E_TIMEOUT, and the grid stays latched in that state.
 * Use it on small grids: the waits of successive CTA waves add up. */
dsp_status dsp_test_withhold_next_copy(dsp_grid *g);

/* Test hook (not in the paper) on the tiling of the grid's evolve launches.
 * Grids whose nx is a multiple of 256 (FP32_MIXED every scheme, FP64 EXACT and
 * STRANG_XY) evolve on row strips: a CTA owns 4 rows x 256 columns and shares
 * the per-step momentum work across them; a launch of one such grid whose last
 * wave of CTAs would be at most half full runs its last strips 2 rows high.
 * tiling = 1: that automatic choice (the default); 0: contiguous 1024-point
 * tiles; 2: row strips, all 4 rows high.  Every tiling gives bitwise the same
 * map and density; the hook exists so that a test can show it. */
dsp_status dsp_test_tiling(dsp_grid *g, int32_t tiling);

/* Copies the raw spinor state (dsp_state_bytes bytes) to the host, or back
 * from the host, with the step cursor, for checkpoint / resume.  Synchronise.
 * Checkpointing only: the paper has no counterpart. */
dsp_status dsp_save_state(dsp_grid *g, void *host_buf, int64_t bytes, int64_t *cursor);
dsp_status dsp_load_state(dsp_grid *g, const void *host_buf, int64_t bytes, int64_t cursor);

/* Frees the grid (and the state if the library allocated it).  NULL is OK.
 * Resource management only: the paper has no counterpart. */
dsp_status dsp_destroy_grid(dsp_grid *g);

/* Static string for a status code (the paper has no counterpart). */
const char *dsp_status_string(dsp_status s);

/* ------------------------------------------------------------------------- */
/* Pulse sampler (host).  Fills the midpoint table of a pulse model so callers
 * need not write their own; any other A(t) can be passed to dsp_set_pulse.   */
/* ------------------------------------------------------------------------- */

#define DSP_PULSE_ZERO 0        /* A = 0                                            */
#define DSP_PULSE_SIN2 1        /* (E0/w) sin^2(pi t/T) (sin wt, eps cos wt)         */
#define DSP_PULSE_GAUSS 2       /* (E0/w) exp(-(t-t0)^2/tau^2) (sin wt, eps cos wt)  */
#define DSP_PULSE_TWO_COLOUR 3  /* sin^2(pi t/T) sum_{k=1,2} (E0/(k w))
                                   (sin(k w t + ph_k), eps cos(k w t + ph_k)),
                                   ph_1 = 0, ph_2 = phase2                           */
#define DSP_PULSE_CONST_FIELD 4 /* A_x = -E0 (t - T/2): constant field E_x = E0      */
#define DSP_PULSE_PAPER 5       /* Sec. IV, Eq. (elec_field): E_x = E0 env(t)
                                   cos(w t + phi), sin^2 rise over pi/(2 Omega_rise),
                                   flat, cos^2 fall over pi/(2 Omega_fall) ending at
                                   T; A_x = -int_0^t E_x                             */

typedef struct {
    int32_t kind;
    int32_t reserved;
    double E0, omega, T, tau, t0, eps, phase2, Omega_rise, Omega_fall, phi;
} dsp_pulse_spec;

/* The midpoint samples of Sec. III, Eq. (approx_time), and the asymptotic
 * A_in, A_out of Sec. II: t_i = 0, t_f = T, dt = T/n_steps.  a_mid: host
 * [n_steps][2] at (n + 1/2) dt; a_in = A(0); a_out = A(T); *dt_out = dt.
 * n_steps >= 1. */
dsp_status dsp_sample_pulse(const dsp_pulse_spec *spec, int64_t n_steps, double *a_mid,
                            double *a_in, double *a_out, double *dt_out);

/* The same for DSP_SCHEME_MAGNUS4 (the higher-order decomposition Sec. III
 * mentions): a_gauss host [n_steps][2][2], A at (n + 1/2 - sqrt(3)/6) dt and
 * (n + 1/2 + sqrt(3)/6) dt, the two Gauss points of each step. */
dsp_status dsp_sample_pulse_gauss(const dsp_pulse_spec *spec, int64_t n_steps, double *a_gauss,
                                  double *a_in, double *a_out, double *dt_out);

/* ------------------------------------------------------------------------- */
/* Serving: a continuous-batching request loop (not in the paper).  Requests
 * (each a whole solve) are queued on submit and admitted FIFO while the device
 * footprint fits the budget and a slot is free; every dsp_server_step advances
 * all admitted requests by up to chunk_steps in ONE batched launch, retires
 * the ones that finished (projection fused, density reduced, map copied to
 * the server's host buffer) and admits more.  A request's result is bitwise
 * the same alone or in any mix.                                              */
/* ------------------------------------------------------------------------- */

typedef struct dsp_server dsp_server;

typedef struct {
    int32_t nx, ny;
    double px_min, px_max, py_min, py_max;
    int32_t precision, scheme, valley;
    int32_t keep_map; /* 1: copy the |c+|^2 map back to host memory at the end */
    int64_t n_steps;
    double dt;
    double a_in[2], a_out[2];
} dsp_request;

#define DSP_REQ_QUEUED 0
#define DSP_REQ_ACTIVE 1
#define DSP_REQ_DONE 2
#define DSP_REQ_FAILED 3
#define DSP_REQ_CANCELLED 4

/* hbm_budget_bytes > 0: admission limit on the sum of device footprints
 * (state + table + map + partial sums) of the active requests; max_active
 * >= 1; chunk_steps >= 1: steps per batched launch, rounded down to a multiple
 * of 16 when it is 16 or more (a request's result is then bitwise the same alone
 * or in any mix, see dsp_evolve).
 * cuda_stream as above. */
dsp_status dsp_server_create(int64_t hbm_budget_bytes, int32_t max_active, int64_t chunk_steps,
                             void *cuda_stream, dsp_server **out);

/* Queues a request; a_mid is its host midpoint table [n_steps][2] (copied).
 * Validation as dsp_create_grid + dsp_set_pulse (DSP_E_CFL included); a
 * request whose footprint alone exceeds the budget is refused (DSP_E_NOMEM).
 * *id receives its id (0, 1, 2, ... in submit order). */
dsp_status dsp_server_submit(dsp_server *s, const dsp_request *req, const double *a_mid,
                             int64_t *id);

/* One scheduling iteration, pipelined: admits what fits, queues one batched
 * launch that advances every admitted request by up to chunk_steps (with the
 * projection, density and result copies of those whose last steps are in it),
 * then waits only for the PREVIOUS iteration and retires the requests that
 * finished there (so the device always has the next iteration queued).  Device
 * memory comes from the stream-ordered pool; nothing blocks on an allocation.
 * Outputs may be NULL: requests admitted and not yet retired, requests still
 * queued, requests retired by this call. */
dsp_status dsp_server_step(dsp_server *s, int32_t *n_active, int32_t *n_queued,
                           int32_t *n_finished);

/* State of a request (DSP_REQ_*), its density once DONE, and (if keep_map)
 * its map copied into map_host (nx*ny doubles or floats by precision; may be
 * NULL).  Steps done so far in *steps_done (may be NULL). */
dsp_status dsp_server_query(dsp_server *s, int64_t id, int32_t *state, double *density,
                            void *map_host, int64_t *steps_done);

/* Cancels a queued or active request; its device memory is freed at the next
 * step.  Other requests are unaffected. */
dsp_status dsp_server_cancel(dsp_server *s, int64_t id);

/* Frees everything.  NULL is OK.  (Like every dsp_server_* call: serving
 * only, the paper has no counterpart.) */
dsp_status dsp_server_destroy(dsp_server *s);

#ifdef __cplusplus
}
#endif

#endif /* DSP_H */
