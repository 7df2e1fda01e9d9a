/*
 * cube.h -- C ABI of libcube: CUBE's information-optimised particle-mesh step
 * (Yu, Pen & Wang, "CUBE: An Information-optimized parallel Cosmological
 * N-body Algorithm") on one NVIDIA GB300 (sm_103a).
 *
 * The library keeps a simulation's particles in the paper's compressed,
 * cell-ordered store (Sections 2.1-2.2; the checkpoint {rho_c, v_c, chi_d,
 * nu_d, I_P} of Section 2.3.1): per-coarse-cell counts rho_c, a coarse
 * velocity field v_c, n_chi-byte fixed-point positions relative to the parent
 * coarse cell (Eqs. chi, x) and n_nu-byte arctan-mapped velocities relative to
 * v_c (Eqs. nu, v).  One cube_pm_step() is one kick + drift of the whole store
 * with a particle-mesh force on the fine mesh, followed by the two-pass
 * re-sort of Fig. update_xp.  Every step of that path runs in the library's
 * own CUDA kernels.
 *
 * Units: lengths in fine mesh cells, time in 1/H0, momentum
 * p = a^2 dx/dt in fine cells x H0, particle mass = N_f^3 / N_p so that the
 * mean density is 1 per fine cell.  Positions are periodic in [0, N_f).
 *
 * Conventions for every entry point:
 *  - Returns CUBE_OK or an error code; nothing throws across the ABI.
 *    cube_last_error() gives a message for the calling thread's last error.
 *  - Array arguments may be host or device pointers; the library asks the
 *    CUDA runtime which one it is.  Host arrays are staged through the
 *    context's stream and the call synchronises before returning; with
 *    device arrays the call only enqueues work on the context's stream,
 *    except where noted.
 *  - The caller owns every array it passes.  The library owns the context
 *    and all device memory inside it (state, scratch, FFT mesh).
 *  - Particle arrays are structure-of-arrays: float pos[3][N] means
 *    pos[0..N) = x, pos[N..2N) = y, pos[2N..3N) = z.
 *  - Errors detected on the device (a particle moving more than one coarse
 *    cell in a step, non-finite input, a count overflow) are latched in a
 *    device flag and returned by the next call that synchronises:
 *    cube_decode, cube_power_spectrum, cube_stats, cube_state_view,
 *    cube_density, cube_potential, cube_debug_drifted.
 *  - One context is one simulation; contexts are independent.  A context
 *    must not be used by two threads at once.
 */
#ifndef CUBE_H
#define CUBE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cube_ctx cube_ctx;

typedef enum {
    CUBE_OK = 0,
    CUBE_E_ARG = 1,        /* invalid argument or unsupported configuration     */
    CUBE_E_NOMEM = 2,      /* a device or pinned-host allocation failed          */
    CUBE_E_CUDA = 3,       /* a CUDA runtime call failed (incl. no device)       */
    CUBE_E_STATE = 4,      /* call out of order, e.g. a step before cube_encode  */
    CUBE_E_MIGRATION = 5,  /* a particle moved more than one coarse cell         */
    CUBE_E_OVERFLOW = 6,   /* non-finite input or a counter overflow             */
    CUBE_E_TIMEOUT = 7     /* a bounded device-side wait (the force pass's tile
                              copy) gave up; the context stays usable        */
} cube_status;

enum { CUBE_GRAD_FD4 = 0 };

typedef struct {
    int32_t n_fine;        /* N_f fine cells per side: 2^a or 3 * 2^a, 16..1024 */
    int32_t ratio;         /* R fine cells per coarse cell (Section 2.3.1): 1, 2,
                              4 or 8, with N_c = N_f / R >= 3                    */
    int64_t n_particles;   /* N_p >= 1 (< 2^31)                                 */
    int32_t x_bytes;       /* n_chi in {1, 2}: position code width (Eq. chi);
                              4 together with v_bytes = 4: uncompressed FP32
                              particles (see "Uncompressed store" below)       */
    int32_t v_bytes;       /* n_nu in {1, 2}: velocity code width (Eq. nu)      */
    int32_t id_bytes;      /* n_I: 0 (no particle IDs), 1, 2 or 4 bytes of I_P
                              per particle (Section 2.1: a PID array tells
                              particle types apart -- 1 byte holds eight kinds
                              as bits, or 256 type numbers -- or every
                              particle); the uncompressed store: 0 or 4      */
    int32_t gradient;      /* CUBE_GRAD_FD4: 4th-order finite-difference force  */
    int32_t deconv_power;  /* the Green's function is divided by W_CIC(k)^p,
                              p in {0, 1, 2}; 2 compensates deposit and gather  */
    int32_t brick;         /* side, in coarse cells, of the storage-order brick:
                              cells are grouped in bricks of brick^3, bricks and
                              cells inside them are x-fastest.  1, 2 or 4 with
                              >= 3 bricks per side and 4 <= brick * R <= 16;
                              0 = automatic: the largest such value            */
    double box;            /* box side L in Mpc/h (units of k and P(k) only)   */
    double omega_m;        /* Omega_m: source term of lap Phi = 1.5 Om (rho-1)  */
    double omega_l;        /* Omega_Lambda: expansion rate E(a)                 */
} cube_params;

/* Uncompressed store (x_bytes = v_bytes = 4): the comparison arm of the
   paper's precision study (Section 3: compressed runs against an
   uncompressed PM code).  The store holds float positions (fine cells, in
   [0, N_f)) and momenta in input order, updated in place; no codes, cells or
   codec scale.  cube_pm_step runs the same mesh part, then per particle a
   CIC gather of the FD4 force, the kick and the drift (periodic).  The
   density is deposited with float atomics, so its last bits depend on the
   summation order.  cube_state_view: chi and nu point to [3][N_p] floats
   (positions, momenta), counts, offsets and vc are NULL, sigma 0.
   cube_keep_drifted(ctx, 1) returns CUBE_E_STATE. */

/* Message describing the calling thread's most recent error ("" if none).
   The pointer stays valid until the thread's next failing call. */
const char* cube_last_error(void);

/* Create a context for one simulation (Section 2.3.3, "initialize": mesh and
   FFT tables, force-kernel factors).  `cuda_stream` is a cudaStream_t (NULL =
   the legacy default stream) on which every later call enqueues its work; the
   current CUDA device at this call is the context's device.  Allocates all
   device memory the context needs: about (2 (3 n_chi + 3 n_nu + n_I) + 45) N_p
   + 8.2 N_f^3 + 78 N_c^3 bytes (both stores, the padded mesh, the ghosted
   potential, histograms, scratch and staging for host arrays; 2.35 GB at
   256^3 particles, 512^3 mesh, x1v1 with IDs).  cube_server_sizes gives the
   exact figures, split into the resident state and the per-call work area.
   Errors: CUBE_E_ARG (params), CUBE_E_NOMEM, CUBE_E_CUDA. */
cube_status cube_create(const cube_params* params, void* cuda_stream, cube_ctx** out);

/* Release the context and its device memory (Section 2.3.3, "finalize").
   Synchronises the context's stream first.  NULL is accepted. */
cube_status cube_destroy(cube_ctx* ctx);

/* Build the compressed store from float particles: the two passes of the
   initial-condition generator (Fig. fig.ic; Section 2.3.2).
   pos   [3][N_p] float, fine-cell coordinates (wrapped periodically);
   vel   [3][N_p] float, momenta p;
   id    [N_p] uint32 particle IDs, or NULL for 0..N_p-1 (ignored if id_bytes=0);
         the low id_bytes bytes of each are stored (cube_decode returns them
         zero-extended);
   a     scale factor of both positions and momenta;
   sigma per-dimension velocity-code scale sigma_Delta/sqrt(3) of Eqs. nu, v
         (Eq. vdelta gives it at the ICs); <= 0 measures it from the particles
         as sqrt(<(v - v_c)^2>).  Either way it is snapped to 2^(m/16).
   Cells are floor(pos / R); within a cell particles keep their input order.
   v_c is the cell mean of vel in 2^-24 fixed point.
   Errors: CUBE_E_ARG, CUBE_E_OVERFLOW (non-finite input, latched), CUBE_E_CUDA. */
cube_status cube_encode(cube_ctx* ctx, const float* pos, const float* vel, const uint32_t* id,
                        double a, double sigma);

/* One particle-mesh step from a_from to a_to (> a_from), KD splitting of the
   (DKKD)^n integrator of Section 2.3.3: positions at a_n = a_from, momenta at
   a_{n-1/2} (at a_n before the first step).  In order: CIC density of the
   store; r2c FFT; times the Green's function -(3/2) Om / k^2 / W(k)^p / N_f^3;
   c2r FFT -> Phi; per particle: decode (Eqs. x, v), CIC gather of -grad Phi
   (FD4), kick by int da/(a^2 E) over [a_{n-1/2}, (a_from + a_to)/2], re-encode
   the kicked velocity against the same v_c (Fig. update_vp); measure
   <(v - v_c)^2> and scale it by the momentum growth g(a_to)/g(a_from) for the
   next store's codec scale (Section 2.2, last paragraph); drift by
   int da/(a^3 E) over [a_from, a_to]; new-cell counts and v_c*; scan;
   stable scatter by new cell with Eq. chi / Eq. nu codes against v_c*
   (Fig. update_xp).  Particles of one new cell stay in old storage order.
   Enqueue-only.  Errors: CUBE_E_STATE (no store, or a_from != the store's a),
   CUBE_E_ARG (a_to <= a_from), CUBE_E_CUDA.  Migration beyond one coarse
   cell is latched (CUBE_E_MIGRATION). */
cube_status cube_pm_step(cube_ctx* ctx, double a_from, double a_to);

/* Decode the store to float particles in storage order (Eqs. x, v).
   pos [3][N_p] fine-cell coordinates, vel [3][N_p] momenta at the store's
   momentum epoch (a_{n-1/2} after a step: see cube_stats.a_p), id [N_p] or
   NULL.  Synchronises.  Errors: CUBE_E_STATE, latched device errors. */
cube_status cube_decode(cube_ctx* ctx, float* pos, float* vel, uint32_t* id);

/* Auto power spectrum of the store's particles (Section 3.2, Eq. cps):
   CIC density on the fine mesh, delta = rho / <rho> - 1, r2c FFT,
   P = L^3 / N_f^6 |delta_k|^2 / W(k)^2 averaged over shells i = 1..n_bins of
   the integer wave-vector length (i - 1/2 <= |n| < i + 1/2), r2c modes
   weighted 2 except on the kx = 0 and kx = N_f/2 planes.
   k, pk, nmodes: [n_bins] doubles (host or device), mean |k| in h/Mpc, P in
   (Mpc/h)^3, weighted mode count.  Overwrites the FFT mesh (the next step
   rebuilds it).  Synchronises.  Errors: CUBE_E_ARG, CUBE_E_STATE. */
cube_status cube_power_spectrum(cube_ctx* ctx, int32_t n_bins, double* k, double* pk, double* nmodes);

/* ---------------------------------------------------------------- time step */

/* Largest |p| over the store's particles and the three axes (momenta as
   decoded, Eq. v).  Synchronises.  Errors: CUBE_E_STATE (no store). */
cube_status cube_max_speed(cube_ctx* ctx, double* p_max);

/* Step-size control (Section 2.3.3: the time increment is limited by the
   particles' velocities): the largest a_to <= a_max for which the fastest
   particle of the current store, drifting with its present momentum,
   moves at most `cells` coarse cells over [a, a_to] (a = the store's
   epoch), i.e. p_max * int_a^a_to da / (a^3 E) <= cells * R fine cells.
   The step's own kick changes the momenta before the drift, so keep
   `cells` below 1 (0.5 leaves a factor 2) to stay within cube_pm_step's
   one-cell migration limit.  Synchronises.
   Errors: CUBE_E_ARG (a_max <= a, cells outside (0, 1]), CUBE_E_STATE. */
cube_status cube_next_epoch(cube_ctx* ctx, double a_max, double cells, double* a_to);

/* Largest force component on the mesh: max over nodes and axes of the 4th-
   order gradient -(8 (Phi(+1) - Phi(-1)) - (Phi(+2) - Phi(-2))) / 12 of the
   potential of the context's last step or cube_potential call (momentum per
   unit kick integral, the units of cube_pm_step's kick).  Each particle's
   force component interpolates these node values with CIC weights, so f_max
   bounds every particle's.  0 before any step or cube_potential.  One pass
   over the mesh (about 0.1 ms at 512^3); synchronises.
   Errors: CUBE_E_STATE (no store). */
cube_status cube_max_force(cube_ctx* ctx, double* f_max);

/* The time step of Section 2.3.3's timestep: the increment is limited by the
   particles' velocities, their accelerations and the cosmic expansion.
   drift_cells in (0, 1]: the fastest particle's drift over the step, with
   its momentum kicked by the largest force component (cube_max_force),
   (p_max + F_max int_{a_p}^{(a + a_to)/2} da / (a^2 E)) int_a^{a_to} da / (a^3 E),
   stays within drift_cells coarse cells (F_max = 0 before any step);
   max_dlna >= 0: ln(a_to / a) <= max_dlna (0: no expansion limit). */
typedef struct {
    double drift_cells;
    double max_dlna;
} cube_step_limits;

/* The largest a_to <= a_max within every limit (bisection on the host's
   integrals; synchronises like cube_next_epoch).  binding (nullable): 0 if
   a_max, 1 if the drift, 2 if the expansion limit set a_to.
   Errors: CUBE_E_ARG (limits out of range, a_max not after the store's
   epoch, no positive step possible), CUBE_E_STATE before cube_encode. */
cube_status cube_next_epoch_limited(cube_ctx* ctx, double a_max, const cube_step_limits* lim, double* a_to,
                                    int32_t* binding);

/* The same bound for given maxima, on the host with no context or GPU:
   positions at epoch a, momenta at a_p (0 < a_p <= a; a_p = a right after
   cube_encode, (a_prev + a) / 2 after a step), fastest momentum component
   p_max >= 0, largest force component f_max >= 0, `ratio` fine cells per
   coarse cell, cosmology (omega_m > 0, omega_l >= 0).  cube_next_epoch_limited
   is this call with the context's cosmology, epochs and measured maxima.
   Errors: CUBE_E_ARG (arguments out of range, no positive step possible). */
cube_status cube_epoch_bound(double omega_m, double omega_l, int32_t ratio, double a, double a_p, double a_max,
                             double p_max, double f_max, const cube_step_limits* lim, double* a_to,
                             int32_t* binding);

/* The host integrals of the KD step (Section 2.3.3) and of the codec-scale
   update (Section 2.2), as cube_pm_step evaluates them; no context or GPU.
   kick = int_{a0}^{a1} da / (a^2 E), drift = int_{a0}^{a1} da / (a^3 E),
   growth_ratio = g(a1) / g(a0) with g = a^2 E f D the linear growth of the
   momenta; E(a)^2 = omega_m a^-3 + (1 - omega_m - omega_l) a^-2 + omega_l.
   EdS (omega_m = 1, omega_l = 0) uses the closed forms, other cosmologies
   Gauss-Legendre quadrature (16 panels of 64 nodes; D from Heath's
   integral).  Outputs may be NULL.  Errors: CUBE_E_ARG (omega_m <= 0,
   omega_l < 0, a0 or a1 <= 0). */
cube_status cube_leapfrog_factors(double omega_m, double omega_l, double a0, double a1, double* kick,
                                  double* drift, double* growth_ratio);

/* ---------------------------------------------------------------- inspection */

typedef struct {
    int32_t n_coarse;        /* N_c                                            */
    int32_t brick;           /* storage-order brick side in coarse cells       */
    int32_t x_bytes, v_bytes, id_bytes;
    int64_t n_particles;
    const uint32_t* counts;  /* device [N_c^3], storage order (rho_c)          */
    const uint32_t* offsets; /* device [N_c^3 + 1], exclusive scan of counts   */
    const float* vc;         /* device [3][N_c^3], storage order (v_c)         */
    const void* chi;         /* device [3][N_p] int8 or int16 (chi_d)          */
    const void* nu;          /* device [3][N_p] int8 or int16 (nu_d)           */
    const uint32_t* id;      /* device [N_p] (I_P) or NULL                     */
    double sigma;            /* per-dimension codec scale of the store         */
    double a;                /* epoch of the positions                         */
    double a_p;              /* epoch of the momenta                           */
} cube_state;

/* Device pointers to the current store (valid until the next cube_pm_step,
   cube_encode or cube_destroy).  Synchronises.  Errors: CUBE_E_STATE. */
cube_status cube_state_view(cube_ctx* ctx, cube_state* out);

typedef struct {
    double mass;             /* total particle mass: (sum of the cell counts,
                                reduced on the device) x N_f^3 / N_p, i.e.
                                N_f^3 for a consistent store; the
                                uncompressed store counts N_p particles      */
    double momentum[3];      /* sum over the current store's particles of the
                                momenta as cube_decode returns them (FP32),
                                each rounded to a multiple of 2^-24 and summed
                                exactly in int64 on the device: within
                                N_p 2^-25 of the exact sum, independent of
                                the summation order                           */
    double sigma;            /* current codec scale                            */
    double a, a_p;           /* epochs of positions and momenta                */
    int64_t steps;           /* cube_pm_step calls since cube_encode           */
    int32_t max_migration;   /* largest |cell shift| of the last step (<= 1)   */
    uint32_t error_flags;    /* bit 0 migration, bit 1 non-finite, bit 2 count,
                                bit 3 a bounded tile-copy wait gave up         */
    double last_step_ms;     /* device time of the last step's kernels         */
    int64_t kernel_launches; /* CUDA kernels this context launched before this
                                call (the call's own reduction not counted)    */
    uint32_t features;       /* bit 0: pass A loads its Phi tiles by TMA
                                (cp.async.bulk.tensor) rather than cp.async   */
} cube_stats;

/* Bookkeeping of Section 2.3.3 (particle count, mass, momentum, codec scale,
   largest migration).  Synchronises.  Returns the latched device error, if
   any, after filling `out`. */
cube_status cube_stats_get(cube_ctx* ctx, cube_stats* out);

/* CIC density of the current store on the fine mesh, rho[z][y][x] floats
   (N_f^3, mean 1).  Overwrites the FFT mesh.  Synchronises.
   Errors: CUBE_E_STATE. */
cube_status cube_density(cube_ctx* ctx, float* rho);

/* Potential Phi[z][y][x] of the current store: density, r2c FFT, Green's
   function with CIC deconvolution, c2r FFT (the mesh part of cube_pm_step).
   Synchronises.  Errors: CUBE_E_STATE. */
cube_status cube_potential(cube_ctx* ctx, float* phi);

/* Keep (1) or stop keeping (0) each step's drifted particles before the
   re-sort, for cube_debug_drifted and cube_debug_force.  Costs 40 bytes per
   particle per step. */
cube_status cube_keep_drifted(cube_ctx* ctx, int32_t enable);

/* Drifted particles of the last step, in the old storage order: the state
   that Fig. update_xp's second loop encodes.
   cell_old [3][N_p] int32 old coarse cell, u_new [3][N_p] float offset in
   coarse-cell units relative to cell_old after the drift, p [3][N_p] float
   kicked momenta (as re-encoded against the old v_c), and *sigma_next the
   codec scale the new store was encoded with.  Synchronises.
   Errors: CUBE_E_STATE (not kept, or no step yet). */
cube_status cube_debug_drifted(cube_ctx* ctx, int32_t* cell_old, float* u_new, float* p,
                               double* sigma_next);

/* Force of the last step at each particle, in the old storage order (the
   order of cube_debug_drifted): F [3][N_p] float = -grad Phi by the 4th-order
   central difference on the fine mesh, interpolated to the particle by CIC
   (the PM force of Section 2.3.3's update_vp, before it is multiplied by the
   kick factor), in the units of the potential: lap Phi = (3/2) Omega_m
   (rho - 1) with lengths in fine cells.  `force` may be host or device
   memory, caller-owned.  Synchronises.
   Errors: CUBE_E_ARG (NULL), CUBE_E_STATE (not kept, or no step yet). */
cube_status cube_debug_force(cube_ctx* ctx, float* force);

/* Self-check of the compact form in which the step kernels read 2-byte
   velocity codes' tables (Eq. v decode values tan(pi k / M) gamma and Eq. nu
   thresholds, Section 2.2): each entry is rebuilt, as the kernels rebuild
   it, from a fixed FP32 approximation and a 4-bit correction, and compared
   with the full table of the current store's codec, for every k in
   [-lim, lim] (decode) and [0, lim + 1] (thresholds).  out2[0] = entries that
   differ (0: the kernels see the exact tables), out2[1] = entries kept as
   "read the full table" (correction out of range).  `out2` is host memory.
   Synchronises.
   Errors: CUBE_E_ARG (NULL, or codes other than 2-byte velocities),
   CUBE_E_STATE (no store). */
cube_status cube_debug_velocity_tables(cube_ctx* ctx, int64_t* out2);

/* ---------------------------------------------------------------- tracing */

/* Kernel phases of one cube_pm_step, in launch order:
   0 setup (clears the new-store counters; no kernel), 1 deposit (CIC density),
   2 fft_x_r2c, 3 fft_y_fwd, 4 fft_z_green (z forward, Green's function, z
   inverse), 5 fft_y_inv, 6 fft_x_c2r, 7 pass_a (decode, force gather, kick,
   drift, per-brick histograms of the new cells), 8 codec (next codec scale
   and tables), 9 scan (of the histograms in cell-major, brick-minor order:
   per-brick starts), 10 cells (new counts, offsets and v_c),
   11 pass_b (stable scatter and encode).  Section 2.3.3 places such timing
   statistics in the code's final stage. */
#define CUBE_PHASES 12

/* Record CUDA events on the context's stream at every phase boundary of the
   next `max_steps` cube_pm_step calls (0 stops recording).  Resets the trace.
   The events are recorded between kernels and do not synchronise.
   Errors: CUBE_E_ARG. */
cube_status cube_profile(cube_ctx* ctx, int32_t max_steps);

/* Per-phase device time summed over the traced steps: ms[CUBE_PHASES]
   (required), kernels[CUBE_PHASES] kernels launched per phase per step (or
   NULL), *nsteps traced steps (or NULL).  Synchronises. */
cube_status cube_profile_read(cube_ctx* ctx, double* ms, int32_t* kernels, int32_t* nsteps);

/* Name of a phase ("" outside 0..CUBE_PHASES-1).  Static storage. */
const char* cube_phase_name(int32_t phase);

/* ---------------------------------------------------------------- allocation-free entry point */

/* Exclusive prefix sum of per-cell particle counts into the offsets of the
   cell-ordered store, without allocating anything.  The paper has no
   counterpart: it exists for callers that cannot call cudaMalloc -- code
   running inside a CUDA-graph capture, under a custom or pooled allocator
   that must own every allocation, or in an embedded runtime with a fixed
   memory budget.
   counts  [n_cells] uint32 device array, read-only;
   offsets [n_cells + 1] uint32 device array, written: offsets[i] = sum of
           counts[0..i), offsets[n_cells] = total (the caller owns both);
   cuda_stream: cudaStream_t to enqueue on (NULL = legacy default stream).
   Scratch: a fixed 256 KiB array in the library's device memory, held by
   every GPU that loads libcube until the process exits; it limits n_cells to
   268,435,456 (CUBE_E_ARG beyond).  The first call on a device looks up the
   array's device address with that device current (make that first call
   before any stream capture).  All calls share the array, so calls that
   overlap on the GPU race with each other; each call writes every scratch
   word it reads, so nothing needs clearing between calls.  Enqueue-only.
   Errors: CUBE_E_ARG, CUBE_E_CUDA (message via cube_last_error). */
cube_status cube_counts_to_offsets_noalloc(const uint32_t* counts, int64_t n_cells, uint32_t* offsets,
                                           void* cuda_stream);

/* ---------------------------------------------------------------- checkpoint */

/* The compressed store as one buffer -- the paper's checkpoint {rho_c, v_c,
   chi_d, nu_d, I_P} (Section 2.3.1), plus the codec scale and the leapfrog
   epochs needed to continue.  Layout (little-endian): a 64-byte header
   {"CUBECKP1", n_fine, ratio, n_particles, x_bytes, v_bytes, id_bytes,
   brick, a, a_p, sigma}, then 16-byte aligned sections: counts u32[N_c^3],
   v_c f32[3][N_c^3], chi [3][N] and nu [3][N] codes of x_bytes / v_bytes,
   ids (id_bytes bytes each) [N] when id_bytes > 0.  The uncompressed store (x_bytes = 4)
   stores positions f32[3][N] and momenta f32[3][N] instead of the first four
   sections.  12 bytes per particle for x1v1 with ids (6 of codes, 4 of
   ids, 2 of coarse fields at 8 particles per coarse cell), against 28 for
   float positions, momenta and ids.

   cube_checkpoint_size: buffer bytes for these parameters (no device needed).
   cube_checkpoint_save: writes the current store into buf (host or device,
   caller-owned, cube_checkpoint_size bytes); synchronises; reports latched
   device errors like cube_decode.
   cube_checkpoint_load: replaces the context's store with the checkpoint in
   buf (host or device); the header's parameters must equal the context's
   (CUBE_E_ARG otherwise, as for a wrong magic, non-positive epochs or codec
   scale, or counts that do not add up to n_particles); rebuilds the offsets
   (scan of the counts) and the codec tables; synchronises.  The next
   cube_pm_step continues from the saved epochs a and a_p.  A load that
   fails after the header checks leaves the context without a store
   (CUBE_E_STATE until the next encode or load). */
cube_status cube_checkpoint_size(const cube_params* params, int64_t* bytes);
cube_status cube_checkpoint_save(cube_ctx* ctx, void* buf);
cube_status cube_checkpoint_load(cube_ctx* ctx, const void* buf);

/* The coarse density field in one byte per cell (Section 2.1): a count below
   255 as itself, 255 for a cell of 255 or more particles, whose count
   follows in `overflow` (4-byte integers, in cell order).  Host arrays;
   no device is needed.
   cube_counts_pack: counts[n_cells] -> bytes[n_cells] and overflow[..];
   *n_overflow receives the list's length; CUBE_E_ARG when it exceeds
   overflow_cap (call again with a list that long).
   cube_counts_unpack: the inverse; CUBE_E_ARG when the 255 bytes and the
   overflow entries do not correspond one to one or an entry is below 255. */
cube_status cube_counts_pack(const uint32_t* counts, int64_t n_cells, uint8_t* bytes, uint32_t* overflow,
                             int64_t overflow_cap, int64_t* n_overflow);
cube_status cube_counts_unpack(const uint8_t* bytes, int64_t n_cells, const uint32_t* overflow, int64_t n_overflow,
                               uint32_t* counts);

/* ---------------------------------------------------------------- memory model */

/* The paper's memory model of one image (Section 2.3, memory layout; Eqs.
   npmax, nptile, Mp_particle, Mp_coarse, Mp_fine and Table t.memory): the
   bytes of each array an image of a multi-image, tiled CUBE run keeps, for
   sizing runs and comparing layouts.  Host only, no device. */
typedef struct {
    int32_t x_bytes, v_bytes;     /* n_chi, n_nu in {1, 2}                          */
    int32_t id_bytes;             /* n_I in {0, 1, 2, 4}                            */
    int32_t ratio;                /* R: fine cells per coarse cell, >= 1            */
    int32_t coarse_per_image;     /* N_c / M_g: coarse cells per image side, >= 1   */
    int32_t buffer;               /* N_b: buffer depth in coarse cells, >= 0        */
    int32_t tiles;                /* M_t: tiles per image side, divides N_c / M_g   */
    double eps_image;             /* inhomogeneity margin of an image, >= 0         */
    double eps_tile;              /* inhomogeneity margin of a tile, >= 0           */
    double particles_per_image;   /* <P_local> > 0                                  */
} cube_memory_config;

/* Bytes per image; divide by particles_per_image for bytes per particle.
   With N_t = (N_c/M_g) / M_t, N_e = N_t + 2 N_b, b = (1 + 2 N_b / N_t)^3,
   P_max = <P_local> b (1 + eps_image) and
   P*_max = <P_local> b (1 + eps_tile) / M_t^3:
     chi_nu      = (3 n_chi + 3 n_nu) P_max      chi_d, nu_d
     chi_nu_tile = (3 n_chi + 3 n_nu) P*_max     chi*_d, nu*_d (tile)
     ids         = n_I (P_max + P*_max)          I_P, I_P*
     rho_c, v_c  = 4, 12 bytes x (N_e M_t)^3     coarse counts and velocities
     k_c         = 12 (N_c/M_g)^3 / 2            coarse force kernel
     k_f         = 12 (R N_e / 2 + 1)(R N_e)^2   fine force kernel of one tile
   The buffer factor in P*_max and the tile-sized K_f are the readings under
   which the equations reproduce Table t.memory (Eq. nptile omits b; Eq.
   Mp_fine's N_t^-3 is garbled).  Arrays that share memory with these
   (F_c, F_f, the FFT work arrays) are not counted, as in the table.
   Errors: CUBE_E_ARG for a NULL pointer or a field out of range. */
typedef struct {
    double chi_nu, chi_nu_tile, ids;
    double rho_c, v_c, k_c;
    double k_f;
    double total;                 /* sum of the rows above                          */
} cube_memory_layout;

cube_status cube_memory_model(const cube_memory_config* cfg, cube_memory_layout* bytes);

/* ---------------------------------------------------------------- autotuning */

/* Picks the storage-order brick (cube_params.brick: 1, 2 or 4 coarse cells)
   that steps fastest for these parameters on this GPU.  The brick is the
   tile shape of the deposit, of the force gather's potential tile and of the
   re-sort; every valid brick gives bit-identical results, so the choice
   changes speed only.  For each valid brick: a context on cuda_stream, an
   encode of pos/vel (as cube_encode, ids by index) at epoch a with codec
   scale sigma, one untimed step, then n_steps (1 .. 100) steps of
   Delta a = 1e-4 a timed with CUDA events.  Blocks until done.
   best_brick: the fastest brick side; ms_per_step (nullable): [3] times for
   bricks 1, 2, 4, -1 where a brick is not valid.
   Errors: CUBE_E_ARG, or any error of the calls above. */
cube_status cube_autotune_brick(const cube_params* params, const float* pos, const float* vel, double a,
                                double sigma, int32_t n_steps, void* cuda_stream, int32_t* best_brick,
                                double* ms_per_step);

/* ---------------------------------------------------------------- batches: many simulations per launch */

/* A batch steps several simulations ("members") of the same geometry with one
   launch per kernel of the step: the members share n_fine, ratio,
   n_particles, the code and id widths, the brick, omega_m, omega_l, gradient
   and deconv_power; only the box may differ.  Every member's state and work
   buffers lie in one device slab at a fixed stride, and each kernel takes the
   member as one more grid dimension, with that member's epochs, kick and
   drift factors from a small per-member table.  This is the paper's
   observation that a step's result does not depend on how the volume is
   tiled (Section 3), applied across simulations: a member's results are
   bit-identical to the same simulation stepped alone.

   Each member is a full cube_ctx (cube_batch_member): encode, decode, P(k),
   statistics, checkpoints and single steps through the ordinary calls, on the
   batch's stream.  Do not cube_destroy a member: cube_batch_destroy frees
   them.  Calls are stream-ordered on the batch's stream; the batch must not be
   used by two threads at once. */
typedef struct cube_batch cube_batch;

/* params: [members] parameter sets (they must agree on everything but the
   box; compressed stores only), members in [1, 4096].  Allocates one slab of
   members x (state + work bytes of one member, cube_server_sizes).
   Errors: CUBE_E_ARG, CUBE_E_NOMEM, CUBE_E_CUDA. */
cube_status cube_batch_create(const cube_params* params, int32_t members, void* cuda_stream, cube_batch** out);

/* Waits for the batch's stream, then frees the members and the slab. */
cube_status cube_batch_destroy(cube_batch* batch);

/* The context of member i (owned by the batch).  Errors: CUBE_E_ARG. */
cube_status cube_batch_member(cube_batch* batch, int32_t i, cube_ctx** out);

/* One KD step of every member i with a_to[i] > a_from[i] (a_from[i] must
   equal the member's epoch); members with a_to[i] <= a_from[i] sit the step
   out.  Members stepped together must have taken the same number of steps
   since they were encoded (a member that sat a step out continues alone with
   cube_pm_step).  Host arrays [members].  Enqueues 16 kernel launches for
   the whole batch (a context stepped alone launches the same kernels once
   per step), 6 of them the mesh half, which is skipped for members whose
   potential cube_batch_solve already enqueued.  For meshes up to 256^3 each
   half is captured as a CUDA graph on the second step with the same store
   parity and number of moving members, and replayed on later ones.  Errors: CUBE_E_ARG,
   CUBE_E_STATE; device errors are latched in each member's flags
   (cube_stats_get). */
cube_status cube_batch_step(cube_batch* batch, const double* a_from, const double* a_to);

/* The mesh half of the next cube_batch_step, enqueued early: the CIC
   density of each flagged member's current store and its potential (the FFT
   Poisson solve of Section 2.3.3's update_vp), which do not depend on the
   step's epochs.  A caller can enqueue it right after a step, while the
   read-back that decides the next epochs (cube_batch_epochs_enqueue) is in
   flight, so that the GPU has work while the host waits.  The next
   cube_batch_step uses these potentials for the members it moves that were
   solved here since their store last changed, and solves any others itself:
   the results are the same either way.  stepping: host array [members],
   non-zero = solve.  Flagged members must have taken the same number of
   steps.  Enqueues 6 launches (none if every flagged member is solved).
   Errors: CUBE_E_ARG, CUBE_E_STATE. */
cube_status cube_batch_solve(cube_batch* batch, const int32_t* stepping);

/* For every member i with a_max[i] above its epoch: the largest a_to[i] <=
   a_max[i] that keeps the member's fastest particle within `cells` coarse
   cells (cube_next_epoch), from one read-back of all members' largest
   momentum; a_to[i] = the member's epoch otherwise.  Synchronises.
   Errors: CUBE_E_ARG (cells not in (0, 1], or a member cannot step), CUBE_E_STATE. */
cube_status cube_batch_next_epochs(cube_batch* batch, const double* a_max, double cells, double* a_to);

/* The same in two halves, so the host need not wait: _enqueue queues every
   member's largest-momentum reduction and its copy into pinned memory behind
   the batch's work so far; _poll returns at once, with *ready 0 while the copy
   is in flight, else *ready 1 and a_to as cube_batch_next_epochs gives it.
   Errors: CUBE_E_ARG, CUBE_E_STATE (poll without an enqueue). */
cube_status cube_batch_epochs_enqueue(cube_batch* batch);
cube_status cube_batch_epochs_poll(cube_batch* batch, const double* a_max, double cells, double* a_to,
                                   int32_t* ready);

/* Kernels cube_batch_step has launched for this batch (all members). */
cube_status cube_batch_launches(cube_batch* batch, int64_t* launches);

/* ---------------------------------------------------------------- serving: many simulations on one GPU */

/* A server runs many independent simulations ("requests") at once on one GPU
   with continuous batching: requests arrive at any time, are admitted in
   arrival order while an HBM budget allows, step concurrently on a few CUDA
   streams (one step of each running request after another, at most two steps
   of a request in flight), and finish with the power spectrum of their final
   store.
   Memory.  Between steps a simulation needs only its compressed store
   (Section 2.3's point: a few bytes per particle) plus codec tables; the
   mesh, the ghosted potential, the step histograms and the encode scratch
   are needed only while one of its calls runs.  A request therefore holds
   its state bytes from admission until cube_server_release, and each stream
   holds one work area, sized for the largest request it has run and shared
   by all requests on that stream.  cube_server_sizes gives both figures.
   The budget bounds the sum of the resident states and the work areas.
   Results.  Every kernel of the step is deterministic, so a request's store
   and P(k) do not depend on what else runs beside it.
   Threading.  A server must not be used by two threads at once.  Calls are
   non-blocking except where noted; the server's clock is seconds since
   cube_server_create (steady clock). */
typedef struct cube_server cube_server;

typedef enum {
    CUBE_REQ_QUEUED = 0,     /* submitted, waiting for memory or a slot           */
    CUBE_REQ_RUNNING = 1,    /* encoded and stepping                              */
    CUBE_REQ_DONE = 2,       /* all steps and the final P(k) completed            */
    CUBE_REQ_FAILED = 3      /* a device error was latched (see error)            */
} cube_req_state;

typedef struct {
    int32_t state;            /* cube_req_state                                    */
    int32_t steps_enqueued;   /* steps handed to the GPU so far                    */
    int32_t n_steps;          /* scheduled steps (waypoints when adaptive)         */
    int32_t max_migration;    /* after completion: largest |cell shift| of a step  */
    double t_submit, t_admit, t_done;   /* server clock; -1 before the event       */
    int64_t state_bytes;      /* device bytes held from admission to release       */
    int32_t error;            /* cube_status of a failed request, else CUBE_OK      */
} cube_request_info;

/* Device bytes of one request with these parameters: its resident state and
   the work area it needs on its stream.  Errors: CUBE_E_ARG as cube_create. */
cube_status cube_server_sizes(const cube_params* params, int64_t* state_bytes, int64_t* work_bytes);

/* budget_bytes: bound on resident states + work areas (device bytes);
   n_streams in [1, 64]: CUDA streams (non-blocking, created by the server);
   max_running >= 1: requests stepping at once (1 = one after another, the
   plain sequential method; admission then waits for the running one). */
cube_status cube_server_create(int64_t budget_bytes, int32_t n_streams, int32_t max_running, cube_server** out);

/* Waits for the server's streams, then frees everything it holds. */
cube_status cube_server_destroy(cube_server* srv);

/* Queues a simulation: initial particles pos[3][N], vel[3][N] (host --
   pinned for an asynchronous upload -- or device arrays) and id[N]
   (nullable) at scale factor epochs[0], codec scale sigma as cube_encode,
   then steps through epochs[1 .. n_steps] (n_steps + 1 values, increasing,
   copied), then P(k) in n_bins bins as cube_power_spectrum.
   max_drift_cells = 0: exactly the n_steps steps epochs[i] -> epochs[i + 1].
   max_drift_cells in (0, 1]: the epochs are waypoints and every step is cut
   as cube_next_epoch does, so that the fastest particle drifts at most that
   many coarse cells (the velocity limit of Section 2.3.3's time step); the
   server reads the largest |p| back asynchronously after each step, so a
   request has one step in flight.
   The caller keeps pos, vel and id valid until the request is DONE or
   FAILED.  Returns a ticket (> 0).
   Errors: CUBE_E_ARG (parameters, n_steps < 1, n_bins outside [1, 2048],
   epochs not increasing, max_drift_cells outside [0, 1]), CUBE_E_NOMEM (the
   request alone exceeds the budget, or pinned result memory). */
cube_status cube_server_submit(cube_server* srv, const cube_params* params, const float* pos, const float* vel,
                               const uint32_t* id, double sigma, const double* epochs, int32_t n_steps,
                               double max_drift_cells, int32_t n_bins, int64_t* ticket);

/* Makes progress without blocking: retires finished requests, hands the next
   steps of running requests to the GPU, admits queued requests that fit.
   n_running, n_queued (nullable): requests in those states afterwards. */
cube_status cube_server_pump(cube_server* srv, int32_t* n_running, int32_t* n_queued);

/* Pumps until every submitted request is DONE or FAILED (blocking). */
cube_status cube_server_drain(cube_server* srv);

cube_status cube_server_info(cube_server* srv, int64_t ticket, cube_request_info* out);

/* P(k) of a DONE request into caller arrays of n_bins doubles (host or device).
   Errors: CUBE_E_STATE before DONE; CUBE_E_ARG for an unknown ticket. */
cube_status cube_server_result(cube_server* srv, int64_t ticket, double* k, double* pk, double* nmodes);

/* Decodes a DONE request's resident store as cube_decode (synchronises with
   the request's stream). */
cube_status cube_server_decode(cube_server* srv, int64_t ticket, float* pos, float* vel, uint32_t* id);

/* Frees a DONE or FAILED request's state and returns its bytes to the budget. */
cube_status cube_server_release(cube_server* srv, int64_t ticket);

/* Device bytes held now: resident states plus work areas. */
cube_status cube_server_bytes(cube_server* srv, int64_t* bytes_in_use);

/* Admission order: CUBE_ADMIT_FIFO (default) admits queued requests in
   arrival order; CUBE_ADMIT_SHORTEST admits the queued request with the least
   remaining work (particles x scheduled steps; ties in arrival order) first,
   which shortens short requests' latency at the expense of long ones.  In
   both, the request chosen next waits for memory and nothing overtakes it.
   Applies from the next admission.  Errors: CUBE_E_ARG. */
enum { CUBE_ADMIT_FIFO = 0, CUBE_ADMIT_SHORTEST = 1 };
cube_status cube_server_set_policy(cube_server* srv, int32_t policy);

/* Test hook for the admission path: the next n allocations of a larger
   stream work area report "out of memory" without calling CUDA.  When a
   work area cannot grow, the stream keeps its current area (its running
   requests continue) and the request being admitted alone ends FAILED with
   CUBE_E_NOMEM.  Not part of the paper (its memory model, Section 2.3, has
   no allocator).  Errors: CUBE_E_ARG (NULL server, n < 0). */
cube_status cube_server_inject_alloc_failures(cube_server* srv, int32_t n);

#ifdef __cplusplus
}
#endif

#endif /* CUBE_H */
