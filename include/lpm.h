/*
 * lpm.h - C ABI of the GB300 stochastic Lagrangian particle model.
 *
 * The method is the one of Molnar, Szakaly, Meszaros, Lagzi, "Air pollution modelling
 * using a graphics processing unit with CUDA" (arXiv:0912.3223): particles released
 * from a point source move by the interpolated wind plus a Gaussian random walk
 * (Sec. 2, Eq. 1-2), decay with the time since emission, deposit stochastically (dry
 * below the mixing height, wet where it rains), become inactive at the domain edge, and
 * every n-th step their decayed masses are summed on a rectangular grid (Sec. 3.2).
 *
 * Conventions for every call:
 *  - Every call returns an lpm_status; nothing throws or aborts across this boundary.
 *    The text of the last failure is available from lpm_last_error().
 *  - The caller owns every buffer it passes. The library copies inputs before
 *    returning (or enqueues the copy on the context stream, see lpm_set_met) and keeps
 *    no caller pointer. The library owns all device memory of a context until
 *    lpm_destroy().
 *  - Work is enqueued asynchronously on the CUDA stream given to lpm_create(). The
 *    read-back calls (lpm_concentration, lpm_deposition, lpm_budget, lpm_particles,
 *    lpm_fixed_state, lpm_sync) synchronise that stream and report device-side errors
 *    (LPM_E_NUMERIC for a non-finite particle position).
 *  - A context is used by one host thread at a time.
 *  - Lengths are SI (m, s), masses are in the unit of the emission rate times seconds.
 */
#ifndef LPM_H
#define LPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lpm_ctx lpm_ctx;

typedef enum {
    LPM_OK = 0,
    LPM_E_INVALID = 1,   /* an argument or the configuration is invalid */
    LPM_E_OOM = 2,       /* a device or host allocation failed */
    LPM_E_CUDA = 3,      /* a CUDA runtime call failed */
    LPM_E_STATE = 4,     /* the call is not allowed in the current state */
    LPM_E_NUMERIC = 5,   /* a particle position became non-finite */
    LPM_E_TIMEOUT = 6    /* a bounded device loop hit its iteration limit (reserved: no
                            kernel waits on another, every loop is bounded by its data) */
} lpm_status;

/* Particle status, bits 28..31 of the particle tag; bits 0..27 hold the release step. */
enum {
    LPM_ACTIVE = 0,
    LPM_UNRELEASED = 1,
    LPM_DEP_DRY = 2,
    LPM_DEP_WET = 3,
    LPM_EXITED = 4
};

/* Indices of lpm_budget()'s output (all masses at the context's current time). */
enum {
    LPM_B_RELEASED = 0,  /* initial mass of every particle released so far */
    LPM_B_AIR_IN = 1,    /* decayed mass of active particles inside the concentration grid */
    LPM_B_AIR_OUT = 2,   /* decayed mass of active particles outside it */
    LPM_B_DRY = 3,       /* mass removed by dry deposition (at the deposition step) */
    LPM_B_WET = 4,       /* mass removed by wet deposition */
    LPM_B_EXITED = 5,    /* mass carried out of the lateral boundary */
    LPM_B_DECAYED = 6,   /* released minus everything above: mass lost to decay */
    LPM_B_N_ACTIVE = 7   /* number of active particles */
};

/*
 * Configuration (Sec. 3.2: the weather grid, the isotope constants, the source and the
 * output grid). Met nodes sit at x0 + i*dx, y0 + j*dy, z_levels[k] (stretched, the
 * "nonlinear" vertical of Sec. 3.2) and times met_t0 + h*met_dt. The concentration
 * grid has cx*cy*cz uniform cells starting at (cx0, cy0, cz0); the deposition grid
 * uses its horizontal cells. Time step k runs from t_k = k*dt to t_{k+1}.
 */
typedef struct {
    int nx, ny, nz;                 /* met nodes, each >= 2; nz <= 64 */
    double x0, y0, dx, dy;
    const double *z_levels;         /* [nz], strictly ascending, read during lpm_create */
    int n_met_t;                    /* number of met time slabs, >= 1 */
    double met_t0, met_dt;
    int cx, cy, cz;                 /* concentration grid cells, each >= 1 */
    double cx0, cy0, cz0, cdx, cdy, cdz;
    double src_x, src_y, src_z;     /* point source of scenario 0 */
    double dt;                      /* time step (s) > 0 */
    int64_t n_steps;                /* run length S; the last step always bins */
    uint64_t seed;                  /* key of the counter-based generator */
    int bin_every;                  /* bin every n-th step (Sec. 3.2), >= 1 */
    double half_life_s;             /* <= 0: no decay */
    double vd_dry;                  /* dry deposition velocity (m/s); 0: off */
    double h_mix;                   /* mixing-layer height (m) */
    double wet_lambda;              /* wet scavenging coefficient (1/s); 0: off */
    double kh_uniform;              /* horizontal K (m^2/s); < 0: gridded K_h field */
    int reflect_ground, reflect_top;
    double z_top;
    int lateral_exit;               /* leaving [x0, x0+(nx-1)dx] x [y0, ...] inactivates */
    int drift_correction;           /* 1: add (dK_z/dz) dt to z (not in Eq. 2) */
    int n_scenarios;                /* 1: plain method; > 1: batched ensemble */
    int64_t max_particles;          /* particle slots over all scenarios */
} lpm_config;

/* Creates a context on the current CUDA device and allocates its device memory.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream). On failure *out = NULL. */
lpm_status lpm_create(const lpm_config *cfg, void *cuda_stream, lpm_ctx **out);

/* Frees the context and all its device memory (synchronises its stream). NULL is a no-op. */
void lpm_destroy(lpm_ctx *ctx);

/* Text of the last failure on this context (or of the last failed lpm_create when ctx
 * is NULL). Valid until the next call on the context. */
const char *lpm_last_error(const lpm_ctx *ctx);

/*
 * Weather slab t_index (time met_t0 + t_index*met_dt), Sec. 3.2 (weather sampled in x,
 * y, z and time by linear interpolation).
 *   uvwk: [nz][ny][nx][4] float = (u, v, w, K_z); required.
 *   kh:   [nz][ny][nx] float K_h, required iff kh_uniform < 0, else must be NULL.
 *   rain: [ny][nx] uint8, nonzero where it precipitates; NULL = no rain in this slab.
 * on_device = 1: the pointers are device pointers (copied on the context stream, the
 * caller keeps them valid until the stream reaches the copy); 0: host pointers. Pageable
 * host memory is copied before the call returns. Page-locked host memory (cudaMallocHost,
 * cudaHostRegister, a pinned tensor; all given pointers) is copied asynchronously on a copy
 * stream of the context, after the work already enqueued on the context stream, so that
 * later hours arrive while earlier ones are computed: the caller keeps those buffers
 * unchanged until the next lpm_sync (or read-back call) returns; lpm_step waits for the
 * hours its steps use.
 */
lpm_status lpm_set_met(lpm_ctx *ctx, int t_index, const float *uvwk, const float *kh,
                       const uint8_t *rain, int on_device);

/*
 * Source and wind perturbation of a scenario (batched ensemble). (x, y, z): release
 * point. wind_offset: NULL or host [n_met_t][2] float (du, dv), a domain-uniform wind
 * offset interpolated in time like the met; copied. Scenario 0 defaults to the config's
 * source and no offset.
 */
lpm_status lpm_set_source(lpm_ctx *ctx, int scenario, double x, double y, double z,
                          const float *wind_offset);

/* Most perturbation modes lpm_set_modes accepts. */
#define LPM_MAX_MODES 4

/*
 * Spatially varying perturbation of the scenarios' weather (the batched ensemble's
 * perturbed meteorology; the paper's weather varies in x, y, z and t, Sec. 3.2): n_modes
 * plane waves of a horizontal streamfunction shared by every scenario, each scenario
 * adding its own realisation (phases and amplitudes, lpm_set_mode_phases) to the wind:
 *   u += p(z) sum_m amp_m eu_m sin(2 pi (fx_m x + fy_m y + phase_m + omega_m t)),
 *   v += p(z) sum_m amp_m ev_m sin(...),
 * with t the step's start time and p linear between the levels like the weather
 * (constant beyond them). modes: host [n_modes][5] (fx, fy (cycles/m), omega (cycles/s),
 * eu, ev); the field is non-divergent when (eu, ev) is perpendicular to (fx, fy).
 * profile: host [nz] scale at the levels. 0 <= n_modes <= LPM_MAX_MODES (0 turns the
 * modes off); every scenario starts with zero amplitudes. Copied; applies to the next
 * lpm_step. Runs in the extended step kernel (1 particle per thread); lpm_adjoint and
 * lpm_receptors reject a context with modes (LPM_E_INVALID). Like the met and the
 * source, the modes are inputs, not part of lpm_save's state.
 * Errors: LPM_E_INVALID for n_modes out of range, NULL or non-finite arrays.
 */
lpm_status lpm_set_modes(lpm_ctx *ctx, int n_modes, const double *modes, const double *profile);

/*
 * A scenario's realisation of the modes of lpm_set_modes: phase (cycles) and amplitude
 * (m/s) of each, host [n_modes] each, copied. Errors: LPM_E_INVALID for a scenario out
 * of range or NULL / non-finite values.
 */
lpm_status lpm_set_mode_phases(lpm_ctx *ctx, int scenario, const double *phase,
                               const double *amp);

/*
 * Continuous release of a scenario (Sec. 3.2: masses are assigned a priori from the
 * emission profile and the particle budget): n_particles particles over steps
 * [first_step, last_step); particle p leaves at step first + floor(p*S/N)
 * (S = last - first) and carries q(h)*dt/n_s, with h = floor(t/q_dt) clamped to
 * [0, n_q-1] and n_s the number of particles leaving at that step. q: host [n_q] rates
 * (mass/s), copied. Scenarios are released once each, in order 0, 1, ..., before the
 * first lpm_step; their particles take consecutive global ids (the generator's key).
 */
lpm_status lpm_release(lpm_ctx *ctx, int scenario, int64_t n_particles, const double *q,
                       int n_q, double q_dt, int64_t first_step, int64_t last_step);

/*
 * Part of a release held by this context (particle-range partitioning across contexts
 * or GPUs): of a release of n_total particles whose particle 0 has global id id_base,
 * this context holds particles [first_particle, first_particle + count). Release steps,
 * masses and the fixed-point scale are those of the whole release, so the integer grids
 * of disjoint ranges add up exactly to the grid of the whole release. lpm_release(...)
 * is lpm_release_range(..., n, 0, n, ..., id_base = sum of earlier releases' n_total).
 * Particles hold their state independently (Sec. 4.2: particles never interact). A
 * scenario of an ensemble held alone (scenario-range partitioning) passes the id_base it
 * has in the ensemble and draws the same numbers. Global ids are 64-bit: id_base >= 0 and
 * id_base + n_total may exceed 2^32 (the generator counter takes both 32-bit halves).
 * Returns LPM_E_INVALID (nothing changed) for n_total < 1, count < 1, a range outside
 * [0, n_total), id_base < 0, an empty or out-of-run step window, negative or non-finite
 * rates, or more particles than max_particles; LPM_E_STATE for a scenario released out
 * of order or twice, or a window that starts before the current step.
 */
lpm_status lpm_release_range(lpm_ctx *ctx, int scenario, int64_t n_total, int64_t first_particle,
                             int64_t count, const double *q, int n_q, double q_dt,
                             int64_t first_step, int64_t last_step, int64_t id_base);

/* Restarts the run at step 0 with the same weather, sources and releases: particles back
 * at their sources (UNRELEASED), grids, deposition, counters and the error word zeroed.
 * Asynchronous. */
lpm_status lpm_reset(lpm_ctx *ctx);

/*
 * Advances every scenario by n steps (Sec. 3.2 main loop; Eq. 1-2): weather sampled at
 * the old position and t_k, displacement u*dt + N(0,1)*sqrt(2*K*dt) per axis,
 * reflection at the ground/top, lateral exit, dry then wet deposition test, and at the
 * end of every bin_every-th step (and of step n_steps-1) the concentration snapshot.
 * Asynchronous. Fails with LPM_E_STATE if a needed met slab is missing, a scenario was
 * not released, or the run would pass n_steps.
 */
lpm_status lpm_step(lpm_ctx *ctx, int64_t n);

/* Current step index k (number of steps taken). */
lpm_status lpm_current_step(const lpm_ctx *ctx, int64_t *k);

/* Last concentration snapshot of a scenario as mass per m^3, [cz][cy][cx] doubles into
 * the caller's host buffer of n_out = cz*cy*cx elements. Synchronises. */
lpm_status lpm_concentration(lpm_ctx *ctx, int scenario, double *out, size_t n_out);

/* Accumulated dry and wet deposition of a scenario as mass per m^2, [cy][cx] doubles
 * each (n_out = cy*cx). Either pointer may be NULL. Synchronises. */
lpm_status lpm_deposition(lpm_ctx *ctx, int scenario, double *dry, double *wet, size_t n_out);

/* Mass budget of a scenario at the current time, out[8] indexed by LPM_B_*.
 * released - decayed = air_in + air_out + dry + wet + exited. Synchronises. */
lpm_status lpm_budget(lpm_ctx *ctx, int scenario, double out[8]);

/* Particle slots [first, first+count) (global ids) to host: xyz [count][3] float and
 * tag [count] (status << 28 | release step); either may be NULL. Synchronises. */
lpm_status lpm_particles(lpm_ctx *ctx, int64_t first, int64_t count, float *xyz,
                         uint32_t *tag);

/*
 * Raw fixed-point state of a scenario for exact checks. Masses are binned as
 * round(m * 2^shift) into 64-bit integers (shift from the scenario's total released
 * mass, below 2^61 units). conc: [cz][cy][cx], dep: [2][cy][cx] (either NULL);
 * counters[16] (may be NULL) = { bin_out, dep_out_dry, dep_out_wet, exited,
 * active_steps, n_bins, air_in, air_out, n_active, dep_total_dry, dep_total_wet,
 * dose_out, species_1_out, species_2_out, species_3_out, 0 }, air_* and n_active as of
 * the last lpm_budget. *shift may be NULL.
 */
lpm_status lpm_fixed_state(lpm_ctx *ctx, int scenario, uint64_t *conc, size_t n_conc,
                           uint64_t *dep, size_t n_dep, int64_t counters[16], int *shift);

/*
 * Device addresses of the same fixed-point state, for a partitioned run that sums its
 * partitions' grids on the device (particles never interact, Sec. 4.2, so the grids of
 * the whole release are the integer sums of the partitions' grids; see
 * lpm_release_range). *conc: [cz][cy][cx] uint64 of the last snapshot; *dep: [2][cy][cx]
 * uint64, cumulative since lpm_reset; counter i of the scenario (the order of
 * lpm_fixed_state's counters; n_bins is not kept on the device) at
 * (*counters)[i * *counter_stride]. Any output pointer may be NULL. The memory belongs to
 * the context until lpm_destroy and must not be written; its contents are those left by
 * the work enqueued so far on the context stream, so readers order themselves after that
 * stream (lpm_sync, or work on the same stream). Errors: LPM_E_INVALID for a scenario
 * out of range.
 */
lpm_status lpm_device_state(lpm_ctx *ctx, int scenario, const uint64_t **conc,
                            const uint64_t **dep, const uint64_t **counters,
                            int64_t *counter_stride);

/* Launch shape of the particle kernels: threads per block (128, 256 or 512), particles
 * per thread (1, 2 or 4) and occupancy variant (0, 1, 2: at most 128, 80 or 64 registers
 * per thread, i.e. 16, 24 or 32 resident warps per SM). Default 512 x 1 x 2. Results do
 * not depend on it. The paper tuned its launch (32 blocks of 256 threads) with the
 * occupancy calculator (Sec. 3.2); here the autotuner picks among these shapes. */
lpm_status lpm_set_launch(lpm_ctx *ctx, int block, int particles_per_thread, int occupancy);

/* Every every_steps steps (at the multiples of every_steps), re-order the released
 * particles of all scenarios in device memory by the weather cell they occupy, so that
 * the threads of a warp gather from neighbouring cells (a layout change only: every
 * particle keeps its id, hence its random numbers, and all results are bit-identical).
 * 0 turns it off; default 60. A change moves every particle back to its home slot first.
 * Needs about 60 bytes of extra device memory per particle slot, allocated at the first
 * sort. The sorts do not keep the map from home slots to sorted places: the first
 * lpm_particles, lpm_particle_velocity, lpm_budget or lpm_save after a sort rebuilds it
 * (one pass over the slots). */
lpm_status lpm_set_sort(lpm_ctx *ctx, int every_steps);

/*
 * Vertical Langevin (velocity-memory) variant of the random walk of Eq. 2 (no paper
 * counterpart: the paper moves particles by Eq. 1-2 only). Each particle carries a
 * turbulent vertical velocity w', updated every step by Thomson's well-mixed model for
 * Gaussian turbulence with sigma_w^2 = K_z / T_L: w' <- w' - w' dt / T_L
 * + (1 + w'^2 / sigma_w^2) d(sigma_w^2)/dz dt / 2 + sqrt(2 sigma_w^2 dt / T_L) n; then
 * z <- z + (w + w') dt. Reflections reverse w'; a particle starts with sigma_w n' at its
 * release step (n' from Philox stream 2, words 0 and 1, Box-Muller). The horizontal motion
 * stays Eq. 2; drift_correction is ignored (the model carries its own drift term). For
 * dt >> T_L the model reduces to the random walk with the same K_z.
 *
 * lpm_set_langevin: on (0/1) and T_L (s, > 0); before the first step or after lpm_reset
 * (LPM_E_STATE otherwise). Allocates 12 bytes per particle slot. Runs with one particle
 * per thread; not supported by lpm_adjoint (LPM_E_INVALID).
 * lpm_particle_velocity: w' (m/s) of slots [first, first+count) to host (0 for deposited or
 * exited particles). Synchronises.
 */
lpm_status lpm_set_langevin(lpm_ctx *ctx, int on, double t_lagr);
lpm_status lpm_particle_velocity(lpm_ctx *ctx, int64_t first, int64_t count, float *w);

/*
 * Decay chain (Sec. 2: released particles "can transform to other species" by
 * radioactive decay, deterministic from the half-lives). The emitted parent (species 0,
 * the configured half_life_s) decays into species 1, which decays into species 2, ...:
 * each particle's amount of species j per unit of emitted parent after a time a is the
 * closed-form solution of the linear rate equations (Bateman), sum_i c_ji exp(-l_i a).
 * The snapshots (every bin_every steps) and the deposition events then also add each
 * daughter's amount to grids of its own; species 0 stays in the usual grids, and the
 * budget, receptors and dosage refer to species 0.
 *
 * lpm_set_decay_chain: n_species in [1, 4] half-lives (s); half_lives[0] must equal the
 * configured half_life_s, 0 (stable) is allowed for the last species only, and the decay
 * rates must be distinct. Call before the first step or after lpm_reset (LPM_E_STATE
 * otherwise); n_species = 1 removes the chain. Allocates 8 bytes per cell, deposition cell
 * and scenario for each daughter.
 * lpm_species: species' concentration [cz][cy][cx] (mass/m^3), dry and wet deposition
 * [cy][cx] (mass/m^2) of the last snapshot / the run so far, and the raw fixed-point grids
 * (same shift as lpm_fixed_state); any pointer may be NULL. Species 0 gives the usual
 * grids. Daughter mass outside the concentration grid at the snapshot is counter 12 + j - 1
 * of lpm_fixed_state. Synchronises.
 */
lpm_status lpm_set_decay_chain(lpm_ctx *ctx, int n_species, const double *half_lives);
lpm_status lpm_species(lpm_ctx *ctx, int scenario, int species, double *conc, double *dry,
                       double *wet, uint64_t *conc_fixed, uint64_t *dep_fixed);

/*
 * K_z inside the step from Eq. 3 (Sec. 2): K_z(z) = k u* z (1 - z/H_z)^2 / Phi_h(z/L),
 * k = 0.4, for 0 < z < H_z and 0 elsewhere, floored at kz_min (m^2/s). The paper leaves
 * Phi_h open: the Businger-Dyer forms 1 + 5 z/L (stable) and (1 - 16 z/L)^(-1/2)
 * (unstable) are used. u*, 1/L and H_z are hourly column fields on the met grid's (y, x)
 * nodes, interpolated like the weather (bilinear in x, y, linear in t); with
 * drift_correction the drift term is the analytic dK_z/dz. The K_z component of the
 * weather records is then ignored.
 *
 * lpm_set_kz_model: model 0 = the gridded K_z of lpm_set_met (default), 1 = Eq. 3
 * (allocates the column buffers: 48 bytes per column and hour). Model 1 runs with one
 * particle per thread and is not supported by lpm_adjoint (LPM_E_INVALID).
 * lpm_set_boundary_layer: hour t_index of the columns, bl [ny][nx][4] float =
 * (u* (m/s) >= 0, 1/L (1/m), H_z (m) > 0, unused), host memory (validated, copied before
 * return) or device memory (on_device != 0, read on the context stream, not validated).
 * Every hour a step touches must be set (LPM_E_STATE otherwise).
 */
lpm_status lpm_set_kz_model(lpm_ctx *ctx, int model, double kz_min);
lpm_status lpm_set_boundary_layer(lpm_ctx *ctx, int t_index, const float *bl, int on_device);

/*
 * Time-integrated concentration ("dosage"): the paper sums the decayed masses on the grid
 * every n-th step, n >= 4, and integrates the snapshots in time as a post-processing
 * (Sec. 3.2), which it notes the GPU could do in a separate kernel (Sec. 4.2). Here the
 * step kernel does it: with every_steps = n > 0, at t_{k+1} for every step k with
 * (k + 1) % n == 0, the decayed mass of each active particle is added, in the same
 * fixed point as the snapshots, to a per-scenario grid of the concentration grid's shape.
 * lpm_set_dosage (re)starts the dosage from the current step: the grid and the
 * out-of-grid counter (dose_out, counter 11 of lpm_fixed_state) are zeroed, and n = 0
 * turns sampling off. lpm_reset zeroes them too. Allocates 8 bytes per cell and scenario
 * at the first call with n > 0.
 *
 * lpm_dosage: out[cz][cy][cx] (n_out = cz*cy*cx) = sum over the samples of the
 * concentration at the sample times times n*dt, i.e. mass * s / m^3; fixed (may be NULL)
 * receives the raw sums of round(m * 2^(shift - b)), shift that of lpm_fixed_state and
 * b = ceil(log2(floor(n_steps / n))) (so that no sum passes 2^61 units); *n_samples (may
 * be NULL) the number of samples taken. LPM_E_STATE if dosage was never enabled.
 * Synchronises.
 */
lpm_status lpm_set_dosage(lpm_ctx *ctx, int every_steps);
lpm_status lpm_dosage(lpm_ctx *ctx, int scenario, double *out, size_t n_out, uint64_t *fixed,
                      int64_t *n_samples);

/*
 * Checkpoint / resume of a run (no paper counterpart; the counter-based draws make the
 * run state small: step index, particles, grids, counters). lpm_save with buf = NULL sets
 * *n to the size needed; otherwise writes the state into the caller's host buffer of *n
 * bytes (synchronises). lpm_load restores it into a context created with the same
 * configuration, weather, sources and releases (checked as far as the sizes go);
 * continuing from a loaded state gives bit-identical results to the uninterrupted run.
 */
lpm_status lpm_save(lpm_ctx *ctx, void *buf, size_t *n);
lpm_status lpm_load(lpm_ctx *ctx, const void *buf, size_t n);

/* Synchronises the context stream and reports device-side errors. */
lpm_status lpm_sync(lpm_ctx *ctx);

/* Instrumentation (no counterpart in the paper). With profiling on, every advance
 * launch is bracketed by CUDA events on the context stream. lpm_stats returns, since
 * the previous lpm_stats call, the number of kernels the context launched, how many of
 * them were advance launches, and their summed device time in ms (0 unless profiling
 * was on); it synchronises the stream and resets the tallies. Pointers may be NULL. */
lpm_status lpm_set_profiling(lpm_ctx *ctx, int on);
lpm_status lpm_stats(lpm_ctx *ctx, int64_t *launches, int64_t *advance_launches,
                     double *advance_ms);

/*
 * Differentiable parameters of the step (adjoint form): k_scale multiplies both
 * diffusivities in Eq. (2) and (bias_u, bias_v) is added to the interpolated wind in
 * Eq. (1). They apply to lpm_step as well. Defaults 1, 0, 0.
 */
lpm_status lpm_set_params(lpm_ctx *ctx, double k_scale, double bias_u, double bias_v);

/* Replaces a released scenario's emission series q[n_q] (rates for bins of the release's
 * q_dt), keeping its particles and release steps (Sec. 3.2: the masses are assigned from
 * the emission profile). Only at step 0 (after lpm_create or lpm_reset). n_q <= 64. */
lpm_status lpm_set_emission(lpm_ctx *ctx, int scenario, const double *q, int n_q);

/*
 * Receptor concentrations of every scenario over a whole run from step 0 (the run state
 * of lpm_step is not touched): C[s][r] = (1/n_s) sum over the steps k with
 * (k+1) % sample_every == 0 of the sum over particles active after step k of
 * m_p G(X_p - x_r), G a 3D Gaussian kernel of width `bandwidth` (m) plus its image below
 * the ground (terms beyond 6 bandwidths are dropped), n_s = floor(n_steps / sample_every).
 * receptors: host [R][3] (x, y, z), 1 <= R <= 256; C: host [n_scenarios][R]. Also stores
 * the states that lpm_adjoint uses (see lpm_set_adjoint_storage). Synchronous. Not with
 * drift_correction.
 */
lpm_status lpm_receptors(lpm_ctx *ctx, const double *receptors, int R, double bandwidth,
                         int sample_every, double *C);

/*
 * Reverse-mode gradient of L = sum_{s,r} dL_dC[s][r] C[s][r] (hand-written adjoint of the
 * step, events frozen, same keyed random numbers): grad [n_scenarios][3 + nq + 3] =
 * (dL/dx_s, dL/dy_s, dL/dh, dL/dq[0..nq-1], dL/dk_scale, dL/dbias_u, dL/dbias_v) per
 * scenario, nq the longest emission series of the context (shorter series leave zeros).
 * Uses the states stored by the last lpm_receptors with the same receptors, bandwidth,
 * sample_every and parameters, else runs that forward first. Synchronous.
 */
lpm_status lpm_adjoint(lpm_ctx *ctx, const double *receptors, int R, double bandwidth,
                       int sample_every, const double *dL_dC, double *grad);

/*
 * Storage of the receptor forward's states for lpm_adjoint. The forward keeps the whole
 * trajectory (16 B per particle and step, from the first release step of each block of
 * 128 particles on, plus 16 B per particle) when that is at most max_bytes and leaves
 * 8 GiB of device memory free; the backward then reads the states back in reverse. With
 * sorting on (lpm_set_sort > 0, the default) the trajectory is kept in 64-step segments
 * over the particles re-sorted at each segment start (about the same size): by weather
 * cell for one scenario, by scenario and then cell tile for several; with sorting off in
 * release order.
 * Otherwise, and always with max_bytes = 0, it keeps a checkpoint every 64 steps (16 B per
 * particle each) and the backward recomputes each 64-step segment from its checkpoint:
 * with sorting on, the segments in the same sorted order into a scratch of two segments'
 * states (2 x 16 B per particle and step of the widest segment, taken only when it fits in
 * free device memory with 8 GiB spare; one segment is recomputed while the other is
 * swept), else each particle's segment in release order. All forms give the same
 * gradients up to the order of the FP64 sums and of the per-segment FP32 partial sums. Default
 * 128 GiB. Drops the held forward. An allocation that fails falls back to checkpoints (no
 * error). lpm_adjoint_storage: *trajectory = 1 when the last receptor forward kept the
 * trajectory, *bytes = device bytes held for the adjoint's states (trajectory, or
 * checkpoints and scratch).
 */
lpm_status lpm_set_adjoint_storage(lpm_ctx *ctx, uint64_t max_bytes);
lpm_status lpm_adjoint_storage(lpm_ctx *ctx, int *trajectory, uint64_t *bytes);

/*
 * The counter-based draws the step consumes (replacing the Mersenne Twister + Box-Muller
 * of Sec. 2): for each i < n, words[4i..4i+3] = Philox4x32-10(key = seed, counter =
 * (pid[i] low, pid[i] high, step[i], stream)) and normals[3i..3i+2] = the three N(0,1)
 * the step derives from them (stream 0). Host buffers, caller-owned; synchronous on the
 * legacy default stream; allocates temporary device memory. Errors: lpm_last_error(NULL).
 */
lpm_status lpm_draws(uint64_t seed, const uint64_t *pid, const uint32_t *step, uint32_t stream,
                     int64_t n, uint32_t *words, float *normals);

/* Largest n lpm_draws_static accepts. */
#define LPM_DRAWS_STATIC_MAX 65536

/*
 * lpm_draws without device allocation (the paper has no counterpart: this is an
 * interface for callers that must not allocate device memory, e.g. applications whose
 * device memory is owned by their own pool or capped by a fixed budget). Same arguments
 * and results as lpm_draws; 0 <= n <= LPM_DRAWS_STATIC_MAX, larger n is rejected with
 * LPM_E_INVALID. Inputs and outputs are staged through one fixed device array in the
 * library (about 2.6 MB, held by every GPU that loads the library until the process
 * exits); the call makes no cudaMalloc, cudaFree or other allocating call. The first
 * call on each device does a one-time set-up: it looks up that array's device address
 * with the device current. Make that first call before any stream capture begins.
 * Synchronous on the legacy default stream. Every call shares the one array, which keeps
 * the last call's contents (each call overwrites what it uses); calls that overlap on the
 * same GPU, e.g. from several host threads, race with each other.
 * Errors: lpm_last_error(NULL).
 */
lpm_status lpm_draws_static(uint64_t seed, const uint64_t *pid, const uint32_t *step,
                            uint32_t stream, int64_t n, uint32_t *words, float *normals);

#ifdef __cplusplus
}
#endif

#endif /* LPM_H */
