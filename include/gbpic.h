/*
 * gbpic.h - C ABI of the GB300 (sm_103a) explicit electromagnetic PIC hot path.
 *
 * The library advances the cycle of KEMPIC-3D (arxiv 2609.16575, section 2.2,
 * Fig. 2) on one GPU:
 *   1. B^{n-1/2} -> B^n            Faraday half step   (section 2.3, Eq. (13))
 *   2. gather E^n, B^n at x^n      staggered CIC       (section 2.5)
 *   3. u^{n-1/2} -> u^{n+1/2}      relativistic Boris  (section 2.4, Eqs. (19)-(20))
 *      x^{n+1} = x^n + dt u / gamma
 *   4. J^{n+1/2}                   zigzag deposit      (section 2.5, Umeda et al. 2003)
 *   5. B^n -> B^{n+1/2}            Faraday half step
 *   6. E^n -> E^{n+1}              Ampere-Maxwell      (section 2.3, Eq. (14))
 * Steps 1 and 5 together equal the full Faraday step and give exactly the
 * centred B^n of Eq. (21) in exact arithmetic.
 *
 * Units (the paper's normalised units, sections 2.3 and 3.1): c = eps0 = mu0 = 1.
 * Grid: n[0] x n[1] x n[2] cells of size d[0..2], periodic in y and z, and in x
 * unless bc_x = 1 (open x: absorbing faces, see pic_grid_desc).
 * Host field arrays are FP64, [component][k][j][i] with i fastest, each component
 * at its Yee location: Ex(i+1/2,j,k) Ey(i,j+1/2,k) Ez(i,j,k+1/2),
 * Bx(i,j+1/2,k+1/2) By(i+1/2,j,k+1/2) Bz(i+1/2,j+1/2,k); J like E.  Each x line
 * holds n[0] values, or n[0] + 1 with an open x (nodes 0..n[0]: the node-located
 * Ey, Ez, Bx include the face x = n[0]; Ex, By, Bz and all of J read 0 there, since
 * the face Ey, Ez follow the Mur condition and no update reads J on that plane).
 * Particle positions are in cell units (X_d = x_d / d_d, 0 <= X_d < n_d).
 *
 * Ownership: the context owns every device buffer it allocates.  Host and device
 * arrays passed in are borrowed for the duration of the call only.  Every entry
 * point returns a pic_status; nothing aborts and device code never prints.
 * Calls that enqueue work (pic_set_fields, pic_load_species, pic_step) are
 * ordered on the context's stream; errors raised by device code surface at the
 * next synchronising call (pic_sync, pic_get_*, pic_diagnostics).
 * A context is not thread safe: one host thread at a time.
 */
#ifndef GBPIC_H
#define GBPIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum pic_status {
    PIC_OK = 0,
    PIC_ERR_ARG = 1,            /* invalid argument (null pointer, bad size, bad species id) */
    PIC_ERR_CFL = 2,            /* dt violates the 3D CFL bound of Eq. (15) */
    PIC_ERR_OOM = 3,            /* device allocation failed */
    PIC_ERR_CUDA = 4,           /* a CUDA runtime call failed; see pic_last_error */
    PIC_ERR_TILE_OVERFLOW = 5,  /* mover or spill buffer full: particles were lost */
    PIC_ERR_SUPERLUMINAL = 6,   /* a particle moved more than one cell in one step */
    PIC_ERR_NAN = 7,            /* a non-finite momentum was produced */
    PIC_ERR_STATE = 8,          /* call out of order (e.g. species before fields) */
    PIC_ERR_TIMEOUT = 9,        /* a bounded device-side wait gave up */
    PIC_ERR_NO_DEVICE = 10      /* no CUDA device, or not an sm_103 device */
} pic_status;

typedef enum pic_precision { PIC_FP32 = 0, PIC_FP64 = 1 } pic_precision;

typedef struct pic_ctx pic_ctx;  /* opaque */

/* Optional device allocator (e.g. a framework's caching allocator).  When alloc
 * is NULL the library uses cudaMalloc/cudaFree. */
typedef void* (*pic_alloc_fn)(size_t bytes, void* user);
typedef void (*pic_free_fn)(void* ptr, void* user);

typedef struct pic_grid_desc {
    int32_t n[3];            /* cells per dimension, >= 1 */
    double d[3];             /* cell sizes (> 0) */
    double dt;               /* time step; must satisfy Eq. (15): dt <= 1/sqrt(sum 1/d^2) */
    double rho_ion;          /* uniform immobile background charge density (diagnostics only) */
    int32_t precision;       /* pic_precision: arithmetic of the whole step */
    int32_t device;          /* CUDA device ordinal */
    void* stream;            /* cudaStream_t to enqueue on; NULL: the library creates one */
    int32_t track_ids;       /* 1: carry each particle's load-order id (pic_get_particles
                                returns load order); 0: tile order, fewer bytes per step */
    int32_t record_every;    /* k > 0: record (U_E, U_B, K) of every k-th step on the device */
    int32_t history_capacity;/* records kept (ring); 0 with record_every > 0 -> 4096 */
    int32_t sort_every;      /* unused (kept for layout): every step writes each tile's particles
                                grouped by cell into the other particle block */
    pic_alloc_fn alloc;      /* optional */
    pic_free_fn free;        /* optional, required when alloc is set */
    void* alloc_user;
    int32_t bc_x;            /* 0: periodic x; 1: open x (boundary modules of section 2.6 as used
                                for the laser wakefield of section 4): first-order Mur on Ey, Ez of
                                the faces x = 0 and x = n[0], particles leaving in x removed */
    int32_t reserved1;
} pic_grid_desc;

/* Soft laser source on an open x (external-source module, section 2.6; section 4):
 * a sheet J_y on the node plane x = plane, J_y = -2 a(t) exp(-r^2 / w0^2) / d[0] with
 * a(t) = a0 exp(-2 ln2 (t - t_peak)^2 / tau^2) sin(omega (t - t_peak)), tau the
 * intensity FWHM and r the distance of the J_y point (y_{j+1/2}, z_k) from (yc, zc)
 * (cell units).  In vacuum the sheet radiates a field of amplitude a(t) to each
 * side; the backward half leaves through the x = 0 face. */
typedef struct pic_laser_desc {
    double a0, omega, w0, tau, t_peak;
    int32_t plane;
    int32_t reserved;
    double yc, zc;
} pic_laser_desc;

/* Moving window on an open x (section 2.2: an operation at the end of the cycle, before
 * the next begins; section 4: the laser-wakefield run moves its window along the
 * pulse).  After every cycle s with s >= start and (s - start) % every == every - 1 the
 * window moves one cell along +x:
 *   - every E and B value takes the value one cell further along x; the new last
 *     value of each x line is zero (the x-node components Ey, Ez, Bx end at the face
 *     x = n[0], the x-half components Ex, By, Bz at x = n[0] - 1/2); J, which the next
 *     cycle recomputes, is not moved (pic_get_fields returns the last cycle's J in the
 *     frame it was deposited in);
 *   - every particle's x cell drops by one (so a particle's position is always relative
 *     to the window); a particle that would be in cell -1 leaves the window and is
 *     counted in n_escaped like one that leaves through a face;
 *   - species `species` receives the plasma of the new last column, at rest
 *     (u^{n+1/2} = 0): a ppc[0] x ppc[1] x ppc[2] lattice per cell at offsets
 *     (2a + 1) / (2 ppc[d]) along each dimension, with weight
 *     density(X) d[0] d[1] d[2] / (ppc[0] ppc[1] ppc[2]), where X is the particle's
 *     absolute x in cells (window cell + moves so far) and
 *     density(X) = density * clamp((X - x0) / ramp, 0, 1) (a step at x0 when ramp = 0);
 *     no particle is made where density(X) = 0.  With track_ids the new particles get
 *     the ids after those loaded, in the order z cell, y cell, z offset, y offset,
 *     x offset (x fastest), move after move.
 * Cell values move exactly (no interpolation); the window moves one whole cell at a
 * time.  every = ceil(d[0] / dt) keeps it at or behind the speed of light. */
typedef struct pic_window_desc {
    int32_t start;        /* first cycle that may end with a move (>= 0) */
    int32_t every;        /* cycles per move (>= 1) */
    int32_t species;      /* index of the species that receives the new plasma */
    int32_t ppc[3];       /* lattice of the new plasma per cell (each >= 1, product <= 4096) */
    double density;       /* plateau density (> 0) */
    double x0, ramp;      /* density profile along absolute x (cells); ramp >= 0 */
} pic_window_desc;

/* Waveguide port on the face x = 0 of an open x (section 3.2: the Yee solver is verified
 * on the TE10 mode of a conducting rectangular guide driven at its input plane).  A hard
 * source: after every Ampere step it sets Ez(0, j, k) = e0 g(t) sin(mode_y pi j / n[1])
 * sin(omega t) and Ey(0, j, k) = 0, with g(t) = 1 - exp(-t / tau) (the start-up envelope
 * of section 3.2) and t the time of the new E; it replaces the Mur condition on that
 * face.  With the wall plane y = 0 (pic_set_pec) the profile is the discrete TE_m0 mode
 * of the guide 0 <= y <= n[1] d[1]. */
typedef struct pic_port_desc {
    double e0, omega, tau;   /* amplitude, angular frequency, envelope rise time (> 0) */
    int32_t mode_y;          /* half waves across y (>= 1) */
    int32_t reserved;
} pic_port_desc;

/* A particle species (section 2.1, Eqs. (8)-(11)): q, m per physical particle;
 * a super-particle of weight w carries q w and m w. */
typedef struct pic_species_desc {
    double q, m;
    int64_t n;                     /* particles */
    const double* X;               /* 3*n: X[0..n) Y[n..2n) Z[2n..3n), cell units, inside the box */
    const double* u;               /* 3*n: u = gamma v (c = 1), same layout */
    const double* w;               /* n weights (> 0) */
    int32_t momenta_at_half_step;  /* 1: u is u^{-1/2}; 0: u is u^0 and the library applies a
                                      backward Boris half step with E^0, B^0 (section 2.4) */
    int32_t device_pointers;       /* 1: X, u, w are device pointers */
    double capacity_slack;         /* tile segment headroom fraction; 0 -> 0.25 */
    int64_t mover_capacity;        /* records of the list of particles changing tile in one step;
                                      0 -> max(n / 4, 65536) (a quarter of the slots with a
                                      moving window).  A step with more movers loses particles
                                      and reports PIC_ERR_TILE_OVERFLOW */
    int64_t spill_capacity;        /* records of the list of movers whose tile segment is full;
                                      0 -> max(n / 16, 65536); overflow as above */
} pic_species_desc;

typedef struct pic_diag {
    int64_t step;            /* steps taken */
    double t;                /* step * dt */
    double U_E;              /* 1/2 dV sum E^n^2 */
    double U_B;              /* 1/2 dV sum B^n^2, B^n = B^{n-1/2} - dt/2 curl E^n (Eq. (21)) */
    double K_half;           /* sum w m (gamma^{n-1/2} - 1) over all species */
    double gauss_max;        /* max_nodes |div E^n - rho^n - rho_ion| (Eq. (2)) */
    double gauss_change_max; /* max_nodes |G^n - G^ref|; G^ref = G at the first pic_diagnostics (taken
                                again at the first call after a moving-window move) */
    double rho_max;          /* max_nodes |rho^n| (electrons + ions) */
    double cont_max;         /* max_nodes |(rho^n - rho^{n-1})/dt + div J^{n-1/2}| (Eq. (12)) when the
                                previous pic_diagnostics call was exactly one step earlier and the
                                window did not move in between, else NaN */
    double J_max;            /* max |J^{n-1/2}| over components and cells */
                             /* (the maxima report +inf when a value they range over is not
                                finite, so a run that blew up cannot show a small residual) */
    int64_t n_alive;         /* particles held, all species */
    int64_t n_spilled;       /* particles currently outside their tile segment (spill list) */
    int64_t n_escaped;       /* particles removed through the open x faces or by the window so far */
} pic_diag;

/* Create a context: validates n, d and the CFL bound of Eq. (15) (section 2.3),
 * allocates the Yee fields (zero) and selects the device.  *out receives the
 * context, or NULL on failure. */
pic_status pic_init_grid(const pic_grid_desc* desc, pic_ctx** out);

/* Set E^0 and B^{-1/2} (section 2.3 time staggering).  E and B each hold 3*N FP64
 * values in the host layout above (N = n0 n1 n2, or (n0 + 1) n1 n2 with an open x);
 * either may be NULL (zero).
 * device_pointers = 1: E, B are device pointers.  Must precede pic_load_species
 * when a species asks for the back-push. */
pic_status pic_set_fields(pic_ctx* ctx, const double* E, const double* B, int32_t device_pointers);

/* Load a species: converts positions to (cell, in-cell offset) in the working
 * precision, sorts particles into 8^3-cell tiles, and applies the backward half
 * push when momenta_at_half_step = 0.  *species_id receives the species index. */
pic_status pic_load_species(pic_ctx* ctx, const pic_species_desc* desc, int32_t* species_id);

/* Set (or, with NULL, remove) the laser sheet of an open x.  PIC_ERR_STATE without
 * bc_x = 1; PIC_ERR_ARG for a plane outside 1..n[0]-1. */
pic_status pic_set_laser(pic_ctx* ctx, const pic_laser_desc* laser);

/* Set the moving window of an open x.  Call it before the species that receives the
 * new plasma is loaded: that species' tile segments are then sized for the plateau
 * density everywhere (a tile fills up as the plasma comes in).  PIC_ERR_STATE without
 * bc_x = 1, after stepping, or when the species is already loaded; PIC_ERR_ARG for
 * out-of-range values.  NULL switches the window off (before stepping only). */
pic_status pic_set_moving_window(pic_ctx* ctx, const pic_window_desc* window);

/* Set the uniform immobile background charge density rho_ion (the value of the grid
 * description; diagnostics only: it enters the Gauss residual and rho_max).  The Gauss
 * reference of gauss_change_max is taken again at the next pic_diagnostics.
 * PIC_ERR_ARG for a non-finite value. */
pic_status pic_set_background(pic_ctx* ctx, double rho_ion);

/* Moves of the window so far (0 without a window). */
int64_t pic_window_moves(const pic_ctx* ctx);

/* Perfectly conducting wall planes (section 3.2 waveguide).  pec_y = 1: the node plane
 * y = 0 conducts, its tangential Ex and Ez are held at zero after every Ampere step; in
 * the periodic y that plane is both walls of a guide 0 <= y <= n[1] d[1] (nothing
 * couples across it).  pec_z = 1: likewise the plane z = 0 (Ex, Ey).  The walls act on
 * the fields only: PIC_ERR_STATE once a species is loaded (and loading a species fails
 * while a wall is set). */
pic_status pic_set_pec(pic_ctx* ctx, int32_t pec_y, int32_t pec_z);

/* Set (or, with NULL, remove) the port of the face x = 0.  PIC_ERR_STATE without
 * bc_x = 1; PIC_ERR_ARG for tau <= 0, mode_y < 1 or non-finite values. */
pic_status pic_set_port(pic_ctx* ctx, const pic_port_desc* port);

/* The current deposit (section 2.5): PIC_DEPOSIT_ZIGZAG (default, the paper's: Umeda et
 * al. 2003) or PIC_DEPOSIT_ESIRKEPOV (Esirkepov 2001, which section 2.5 names among the
 * charge-conserving schemes), both with the first-order (CIC) particle shape and exact
 * discrete continuity.  For a move inside one cell they give the same current (the
 * exact flux of the straight segment through the trilinear cloud); a move across cell
 * faces is one straight segment for Esirkepov (weights Wx = DSx (S0y S0z + DSy S0z / 2 +
 * S0y DSz / 2 + DSy DSz / 3) on the 3x3x3 support, Jx the running sum of -q w Wx /
 * (dt dy dz) along x) and two relayed segments for ZigZag.  The adjoint supports ZigZag
 * only (PIC_ERR_STATE).  Call before stepping or between steps.  The first Esirkepov
 * step of a species reserves device memory for its crossers' records, 40 bytes (FP32)
 * or 80 bytes (FP64) per particle slot; that step returns PIC_ERR_OOM when it cannot. */
typedef enum pic_deposit { PIC_DEPOSIT_ZIGZAG = 0, PIC_DEPOSIT_ESIRKEPOV = 1 } pic_deposit;
pic_status pic_set_deposit(pic_ctx* ctx, int32_t deposit);

/* The particle shape (section 2.5, Eq. (16); section 5 lists higher-order shapes as an
 * extension): PIC_SHAPE_CIC (default, the paper's zeroth-order cloud b0: first-order
 * CIC interpolation and the deposit pic_set_deposit selects) or PIC_SHAPE_TSC (the
 * first-order cloud b1: quadratic B-spline weights W2(r) = 3/4 - r^2 for |r| <= 1/2,
 * (3/2 - |r|)^2 / 2 for 1/2 <= |r| <= 3/2).  With TSC every field component is
 * interpolated from its own Yee location with its 27 nearest samples, the current is
 * Esirkepov's with the same shape on the 4 x 4 x 4 nodes a move touches (whatever
 * pic_set_deposit says), the back-push gathers with TSC, and pic_diagnostics takes the
 * node charge with TSC, so continuity and Gauss's law hold exactly as with CIC.  TSC
 * needs a periodic box without conducting walls (PIC_ERR_STATE for bc_x = 1 or walls
 * set, and pic_set_pec fails while TSC is set); the adjoint and
 * pic_gauss_check_static support CIC only (PIC_ERR_STATE).  Call before stepping or
 * between steps; PIC_ERR_ARG for another value. */
typedef enum pic_shape { PIC_SHAPE_CIC = 1, PIC_SHAPE_TSC = 2 } pic_shape;
pic_status pic_set_shape(pic_ctx* ctx, int32_t shape);

/* Compensated binomial current filter.  Section 2.2 counts "compensated smoothing"
 * among the operations of a cycle and section 2.6 lists a current-filtering module;
 * the paper gives no scheme and its runs use none, so it is off by default.  With
 * passes > 0, each cycle filters the particles' current J^{n+1/2} after the deposit and
 * before the laser sheet and Ampere's law: along x, y and z in turn, one convolution of
 * every component with `passes` binomial stencils (1/4, 1/2, 1/4) and, when
 * compensate = 1, the compensator (-p/4, 1 + p/2, -p/4), p = passes.  A Fourier mode of
 * wave number k_d is multiplied by prod_d (1 - s_d)^p (1 + p s_d), s_d = sin^2(k_d d_d / 2)
 * (without the compensator: prod_d (1 - s_d)^p).  Periodic dimensions wrap; along an open
 * x the values x = 0 .. n[0] - 1 are filtered with zero outside them.  The filtered J no
 * longer satisfies the discrete continuity equation (cont_max reports how far).
 * Allocates a second J set (3 N values) on the first filtered cycle.  PIC_ERR_ARG unless
 * 0 <= passes <= 8 and compensate is 0 or 1; passes = 0 switches it off.  The adjoint
 * refuses a filtered context (PIC_ERR_STATE). */
pic_status pic_set_current_filter(pic_ctx* ctx, int32_t passes, int32_t compensate);

/* Advance nsteps cycles (section 2.2, Fig. 2), asynchronously on the context's
 * stream.  J of the last cycle is kept for pic_get_fields and pic_diagnostics.  In a
 * periodic box without walls, laser, port or moving window, and with neither the energy
 * history nor pic_set_timing on, a call of 6 or more cycles runs its middle cycles as a
 * CUDA graph of two cycles captured once per call and launched repeatedly (the same
 * kernels and results, fewer launch gaps); otherwise every kernel is launched directly. */
pic_status pic_step(pic_ctx* ctx, int32_t nsteps);

/* Wait for the context's stream; returns the first device-side error raised. */
pic_status pic_sync(pic_ctx* ctx);

/* Copy E^n, B^{n-1/2} and J^{n-1/2} out (3*N FP64 values each, host layout above);
 * any pointer may be NULL.  Synchronises. */
pic_status pic_get_fields(pic_ctx* ctx, double* E, double* B, double* J, int32_t device_pointers);

/* Copy one species out as 7 rows of *n FP64 values: X, Y, Z (cell units), ux, uy,
 * uz, w.  With track_ids the rows are in load order (*n = the number loaded, plus the
 * number a moving window has injected; a particle removed through an open x face or
 * by the window reads as NaN in every row), else in tile order (*n = the number
 * alive).  out may be NULL to query *n.  Synchronises. */
pic_status pic_get_particles(pic_ctx* ctx, int32_t species, double* out, int64_t* n, int32_t device_pointers);

/* Checkpoint / resume.  pic_save_state writes the dynamical state to a host byte blob
 * that the library allocates (*blob; *bytes its size; release it with pic_free_state):
 * E^n and B^{n-1/2}, every species' particles held (positions, u^{n-1/2}, weights, and
 * with track_ids their ids), their charge, mass, fixed-point J unit and counters
 * (loaded, injected, escaped), the step count and the window's moves.  Synchronises.
 * pic_load_state restores it into a fresh context (no species loaded, no step taken)
 * created with the same grid, time step, precision, bc_x and track_ids; settings that are
 * not state (laser, window, filter, walls, port, deposit, energy recording) are set on the
 * new context by the caller first, the window before pic_load_state.  The particles are
 * sorted into tiles again, so the run continues as if it had not stopped up to the
 * rounding of the current's partial sums, which follow the particles' order in the tiles.
 * PIC_ERR_ARG for a blob of another configuration or a damaged one, PIC_ERR_STATE for a
 * context that is not fresh. */
pic_status pic_save_state(pic_ctx* ctx, void** blob, size_t* bytes);
void pic_free_state(void* blob);
pic_status pic_load_state(pic_ctx* ctx, const void* blob, size_t bytes);

/* FP64 device reductions of the current state (section 3.3 diagnostics).
 * Synchronises. */
pic_status pic_diagnostics(pic_ctx* ctx, pic_diag* out);

/* Energy history recorded while stepping (record_every > 0): 3 FP64 values per
 * record, (U_E^n, U_B^n, K^n) with K^n = sum w m ((gamma^{n-1/2} + gamma^{n+1/2})/2 - 1),
 * oldest first.  *count receives the number of records written to out. */
pic_status pic_get_history(pic_ctx* ctx, double* out, int32_t max_records, int32_t* count);

/* Per-kernel timing with CUDA events on the context's stream.  enable = 1 starts
 * accumulating; pic_kernel_times returns, for up to max entries, the kernel class
 * name, number of launches and total milliseconds.  Synchronises.  While timing is on,
 * pic_step launches every kernel directly (no graph replay: one event pair per launch). */
pic_status pic_set_timing(pic_ctx* ctx, int32_t enable);
pic_status pic_kernel_times(pic_ctx* ctx, int32_t max, const char** names, int64_t* launches, double* ms,
                            int32_t* count);

/* Bound on the tile kernel's wait for its TMA-staged field boxes, in polls of the
 * mbarrier (each poll may suspend the thread for a short, hardware-defined time).  The
 * default (a negative value restores it) is 2^24 polls; 0 gives up without waiting.  A
 * tile whose wait gives up still waits (bounded) for its copies in flight, then drops its
 * particles; the next synchronising call returns PIC_ERR_TIMEOUT and the context's state
 * is no longer valid (destroy it).  The bound exists so that a stalled copy becomes an
 * error status instead of a hung device, and so that this path can be exercised; it
 * applies to every tile kernel launched after the call.  PIC_ERR_ARG for a null ctx. */
pic_status pic_set_wait_limit(pic_ctx* ctx, int32_t polls);

/* Differentiation: a hand-written discrete adjoint of the cycle of section 2.2.
 * The loss is the field energy of the final state, L = U_E + U_B at time level N
 * (E^N and B^N of Eq. (21)), as in pic_diagnostics.
 *
 * pic_adjoint_forward advances nsteps cycles from the current state s^0, keeping a
 * device-memory snapshot of the full state every ckpt_every steps, and returns L.
 * Needs track_ids = 1 (gradients are reported per loaded particle).  It reserves, in
 * one device allocation, the checkpoints, min(nsteps, ckpt_every) recomputed states and
 * the backward pass's buffers (PIC_ERR_OOM if that fails), so that the backward pass
 * allocates nothing; the reservation lives until the next pic_adjoint_forward or
 * pic_destroy.
 *
 * pic_adjoint_backward returns, for that L,
 *   dL_du[s]: for each species s (an array of species pointers, entries may be
 *             NULL), 3*n_s FP64 values: dL/du^{-1/2} in load order, rows ux, uy, uz;
 *   dL_dA:    <lambda_E^0, E_dir> + <lambda_B^{-1/2}, B_dir>, i.e. dL/dA when the
 *             initial fields are E^0 = A E_dir and B^{-1/2} = A B_dir (E_dir, B_dir:
 *             3*N FP64 values in the host field layout, either may be NULL).
 * It restores each checkpoint, recomputes the segment's states and runs the adjoint
 * kernels (Yee^T, deposit^T, position^T, Boris^T, gather^T) in reverse; the field
 * adjoints and parameter-gradient sums are FP64, the per-particle Jacobian products
 * run in the context's precision.  Afterwards the context holds the final state s^N
 * again.  device_pointers = 1: E_dir, B_dir and dL_du are device pointers.
 * PIC_ERR_STATE without a preceding pic_adjoint_forward, or when a species was loaded
 * since.  Synchronises. */
pic_status pic_adjoint_forward(pic_ctx* ctx, int32_t nsteps, int32_t ckpt_every, double* loss);
pic_status pic_adjoint_backward(pic_ctx* ctx, const double* E_dir, const double* B_dir, double* dL_dA,
                                double* const* dL_du, int32_t device_pointers);

/* pic_adjoint_forward followed by pic_adjoint_backward in one call: the loss and its
 * gradients for the next nsteps cycles from the current state (same arguments and
 * errors as the two calls). */
pic_status pic_adjoint_run(pic_ctx* ctx, int32_t nsteps, int32_t ckpt_every, const double* E_dir, const double* B_dir,
                           double* loss, double* dL_dA, double* const* dL_du, int32_t device_pointers);

/* Allocation-free Gauss check.  The paper has no counterpart: this entry point exists
 * for callers that cannot allocate device memory, e.g. an application whose memory
 * pool already owns the device memory it may use, or a monitoring hook that must not
 * trigger the device-wide synchronisation cudaMalloc/cudaFree can cause while other
 * streams are busy.  It computes the same two values as the gauss_max and rho_max
 * fields of pic_diagnostics (FP64 cloud-in-cell charge of every species on the nodes;
 * max |div E - rho - rho_ion| and max |rho + rho_ion|) but keeps the node charge in a
 * static device array of the library instead of memory it allocates:
 *   - at most 1,048,576 cells (2^20, e.g. 128 x 128 x 64); a larger grid returns
 *     PIC_ERR_ARG with the reason in pic_last_error;
 *   - the array (8 MB) is held until the process exits by every GPU on which a
 *     context was created: pic_init_grid looks up its device address
 *     (cudaGetSymbolAddress, with that device current), which loads the library's
 *     module there and commits the array, so this entry point itself triggers no
 *     module load; called for a device without a context it returns PIC_ERR_STATE;
 *   - all calls share the array and it keeps the last call's contents; each call
 *     clears what it uses, but calls whose work overlaps on the GPU race on it.
 * It calls no cudaMalloc or cudaFree and allocates nothing through the context's
 * allocator.  Synchronises. */
pic_status pic_gauss_check_static(pic_ctx* ctx, double* gauss_max, double* rho_max);

/* Measurement utility (the paper has no counterpart): the FP64 fused multiply-add rate
 * of the given device in FLOP/s (2 per FMA), from a kernel of independent FMA chains
 * timed with CUDA events (about 0.1 s; synchronises the device's default stream).
 * PIC_ERR_ARG for a null output, PIC_ERR_NO_DEVICE without that device. */
pic_status pic_probe_fp64_rate(int32_t device, double* flops_per_s);

/* Total kernel launches the library has issued on this context. */
int64_t pic_launch_count(const pic_ctx* ctx);

/* Human-readable detail of the last error on ctx (never NULL). */
const char* pic_last_error(const pic_ctx* ctx);
const char* pic_status_string(pic_status s);

/* Release every device buffer and the stream the library created. */
void pic_destroy(pic_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* GBPIC_H */
