/*
 * npsim.h -- C ABI of the GB300 (sm_103a) Langevin-dynamics nanoparticle
 * aggregation library.
 *
 * The library advances N nanoparticles (NPs) of up to NPSIM_MAX_TYPES types
 * inside an evaporating or condensing droplet, following the six-step loop of
 * arXiv 2501.04456 Sec. 2.2: (i) binning into cells, (ii) Lennard-Jones and
 * Coulomb pair forces, (iii) the droplet radius, (iv) the interface (surface
 * tension) force, (v) gravity, viscosity and centrifugal force, (vi) the
 * velocity and position update with Brownian noise.  All compute runs in the
 * library's CUDA kernels; this header uses only plain C types.
 *
 * Units are reduced: length = sigma of the reference NP, energy = kT_ref = 1.
 *
 * Conventions shared by every entry point:
 *  - Return value: NPSIM_OK (0) or a negative NPSIM_ERR_* code.  Nothing aborts,
 *    traps or exits; npsim_last_error() gives a message for the calling thread.
 *  - Host arrays of positions, velocities and forces are row-major n x 3
 *    float64 ("xyz xyz ...").  Types are int32 in [0, n_types).
 *  - The caller owns every buffer it passes; the library copies what it keeps.
 *    The library owns the simulation object and its device memory.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *    queued on it; functions that return host data synchronise it.
 *  - A simulation object may be used by one host thread at a time.
 */
#ifndef NPSIM_H
#define NPSIM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NPSIM_MAX_TYPES 8
#define NPSIM_MAX_SCALES 32

enum {
    NPSIM_OK = 0,
    NPSIM_ERR_INVALID_ARG = -1, /* bad size, pointer, type index or parameter */
    NPSIM_ERR_CUDA = -2,        /* a CUDA runtime call failed (message says which) */
    NPSIM_ERR_NONFINITE = -3,   /* a position became NaN/Inf during npsim_step */
    NPSIM_ERR_TIMEOUT = -4,     /* a bounded device-side wait gave up */
    NPSIM_ERR_OOM = -5,         /* device allocation failed */
    NPSIM_ERR_IO = -6,          /* checkpoint file could not be written or read */
    NPSIM_ERR_NO_DEVICE = -7,   /* no CUDA device, or not an sm_103 device */
    NPSIM_ERR_ESCAPED = -8      /* with the full interface spring on (wall 1), an NP was
                                   farther than twice the larger of R0 and R(t) from the
                                   droplet centre: a step went unstable (the paper has
                                   no such check; its runs rely on strong damping) */
};

/* Per-type NP properties (Sec. 2.1: each NP type has its own size, mass and
 * charge, and its own interface spring constant; friction from Stokes' law). */
typedef struct {
    double sigma;  /* diameter; LJ length of the like pair; radius = sigma/2 */
    double eps;    /* LJ well depth of the like pair */
    double mass;
    double charge; /* in units of the elementary charge */
    double gamma;  /* Langevin friction rate (1/time): drag force = -mass*gamma*v */
    double k_wall; /* interface spring constant */
} npsim_type_t;

/* Scenario parameters. */
typedef struct {
    int32_t n_types;    /* 1 .. NPSIM_MAX_TYPES */
    int32_t rot_mode;   /* centrifugal force: 0 none, 1 rotation about z, 2 isotropic */
    int32_t lj_mode;    /* LJ: 0 off, 1 inside the all-pairs kernel, 2 cell list */
    int32_t coulomb;    /* 0 off; 1 all-pairs Coulomb (not truncated); 2 Coulomb truncated
                           (not shifted) at coulomb_cut * sigma_ab, summed with LJ from
                           the cell list (needs lj_mode 2; the paper prints 4 sigma_ab) */
    int32_t wall;       /* interface spring (Sec. 2.2 iv): 0 off (bulk liquid); 1 on every
                           NP beyond its equilibrium point R(t) - r_i; 2 only within
                           the band (-r_i, r_i) about the surface, as step (iv) prints it */
    int32_t integrator; /* 0: BAOAB Langevin; 1: overdamped (Brownian dynamics); 2: the
                           step (vi) as printed: v += dt (F/m - gamma v), then a random
                           velocity of magnitude v_kick in a uniform direction, x += dt v */
    int32_t sum_neutral;  /* 0 (default): NPs of charge 0 are left out of the all-pairs
                             Coulomb sum, whose terms for them are exactly zero (the
                             forces are those of the full sum, up to float32 summation
                             order); 1: sum the Coulomb term over all N(N-1) pairs */
    int32_t reserved_;    /* set to 0 */
    uint64_t seed;      /* Philox key of the noise */
    double dt;          /* time step */
    double kT;          /* temperature of the noise */
    double R0;          /* droplet radius at t = 0 */
    double k_evap;      /* radius-square law R(t)^2 = R0^2 - k_evap*t */
    double g;           /* gravity along -z: force -mass*g */
    double omega;       /* rotation rate of the centrifugal force */
    double bjerrum;     /* Coulomb prefactor C: U = C q_a q_b / r */
    double lj_cut;      /* LJ cutoff in units of sigma_ab (2.5 typical) */
    const double *eps_override; /* n_types x n_types LJ eps matrix, or NULL for
                                   Lorentz-Berthelot eps_ab = sqrt(eps_a eps_b) */
    double v_kick;      /* integrator 2: magnitude of the random velocity added each step */
    double coulomb_cut; /* coulomb 2: Coulomb truncated (not shifted) at coulomb_cut * sigma_ab */
} npsim_params_t;

typedef struct npsim_sim *npsim_sim_t;

/* Message of the last failed call on this thread ("" if none). */
const char *npsim_last_error(void);

/* Library version string and the device it runs on.  sm_count/clock_khz may be NULL. */
int npsim_device_info(int *sm_count, int *clock_khz, int *cc_major, int *cc_minor);

/*
 * Create a simulation of n NPs (Sec. 2.1 starts from NPs placed at random
 * inside the droplet sphere; the caller supplies the initial state so that
 * runs are reproducible).  x0: n x 3 positions; v0: n x 3 velocities or NULL (zero);
 * type: n type indices.  Pair parameters follow Lorentz-Berthelot mixing,
 * sigma_ab = (sigma_a + sigma_b)/2, unless params->eps_override is set
 * (Table 1 prints such a matrix).  The initial total force F(x0, t=0) is
 * computed before returning.  On success *out owns device memory until
 * npsim_destroy.  Errors: INVALID_ARG (n < 1, n > 2^31-1, bad type index,
 * non-positive mass/sigma/dt), OOM, CUDA, NO_DEVICE.
 */
int npsim_create(const npsim_type_t *types, const npsim_params_t *params, int64_t n,
                 const double *x0, const double *v0, const int32_t *type,
                 void *stream, npsim_sim_t *out);

/* Release the object and its device memory (NULL is ignored). */
void npsim_destroy(npsim_sim_t sim);

/*
 * Advance n_steps steps of the loop of Sec. 2.2 (steps i-vi): cell binning (if
 * lj_mode == 2), pair forces, R(t) by the radius-square law, interface spring,
 * gravity, centrifugal force and the Langevin update with Philox4x32-10 noise
 * keyed by (seed) and counted by (particle, step, 0).  Steps are replayed from
 * captured CUDA graphs.  Returns after one device-to-host read of the error
 * word: NONFINITE if any position became non-finite, TIMEOUT if a bounded wait
 * expired, ESCAPED if (wall 1) an NP was farther than 2 max(R0, R(t)) from the
 * centre during some step.  The steps were taken in every case; the word is
 * cleared by the read.  n_steps = 0 is a no-op.
 */
int npsim_step(npsim_sim_t sim, int64_t n_steps);

/* Run n_steps steps and record every `every`-th frame (Sec. 2.2: only every
 * j-th frame of a fine-step run is recorded): after steps every, 2 every, ...
 * the float32 position mirror (x, y, z hi words, charge) of all NPs goes to
 * frames[k] (host, n_frames x n x 4 floats, caller-owned), copied by a side
 * stream from a device staging ring while the next steps compute.  frames is
 * registered as page-locked memory for the call unless it already is.
 * n_frames >= n_steps / every.  Returns after the last frame has arrived and
 * the error flags were read, as npsim_step.  Errors: as npsim_step,
 * INVALID_ARG (every < 1, frames too short). */
int npsim_step_record(npsim_sim_t sim, int64_t n_steps, int64_t every, float *frames,
                      int64_t n_frames);

/* Copy the state to host arrays (any may be NULL): x, v (n x 3), F (n x 3 total
 * force at x and the current time), *step (steps taken since t = 0).  On the
 * device a position is kept as a pair of float32 words (hi + lo, about 48
 * significant bits), a velocity as float32 and a force as a float32 (hi, lo)
 * pair; x and F are returned as the float64 sums of their pairs. */
int npsim_get_state(npsim_sim_t sim, double *x, double *v, double *F, int64_t *step);

/* Replace the state (x required, v may be NULL = zero) and set the step counter;
 * recomputes F at the new positions. */
int npsim_set_state(npsim_sim_t sim, const double *x, const double *v, int64_t step);

/* Forces at the current state into host F (n x 3).  what = 0: total force (pair +
 * external, the one the integrator uses); 1: pair forces only (step ii);
 * 2: LJ only; 3: Coulomb only. */
int npsim_forces(npsim_sim_t sim, int what, double *F);

/* Float32 mirror of the positions (x, y, z, charge) into a caller-owned device
 * buffer of 4*n floats on the simulation's stream (no host synchronisation). */
int npsim_positions_device(npsim_sim_t sim, float *dev_xyzq);

/* Statistics of Sec. 3 at the current state. */
typedef struct {
    double r_max;       /* RDF range (bins cover [0, r_max)) */
    int32_t n_bins;     /* RDF bins (> 0) */
    int32_t radial_bins;/* bins of the radial concentration over [0, R(t)) (0 = skip) */
    int32_t boxcount;   /* 1: compute the box-counting dimension */
    int32_t max_scales; /* box-counting scales d*2^k, k < max_scales (<= NPSIM_MAX_SCALES) */
} npsim_stats_cfg_t;

typedef struct {
    double R;        /* droplet radius R(t) */
    double d_mean;   /* number-mean NP diameter */
    double Rg;       /* radius of gyration (Eqs. Rg, r0) */
    double Df_rg;    /* D_f from the fractal equation (Eq. N, k_f = 1.593) */
    double Df_box;   /* box-counting D_f (NaN if fewer than two scales fit) */
    double center[3];/* centre of mass r0 */
    int32_t n_scales;
    int32_t pad_;
    int64_t nbox[NPSIM_MAX_SCALES];
    int64_t n_surf;  /* NPs at the surface: | |x_i| - R(t) | < r_i (Sec. 1, Sec. 2.2 (iv)) */
} npsim_stats_t;

/*
 * RDF of Sec. 3.2, g(r) = sum_i (psi_i(r)/N) / ((N-1) dV_r / V) with V the
 * droplet volume 4 pi R(t)^3 / 3: pair counts (ordered pairs, int64[n_bins])
 * and g (float64[n_bins]); the radial concentration C_NPs about the droplet
 * centre (Sec. 3.2) into radial_counts/radial_c (int64/float64[radial_bins],
 * both may be NULL); R_g and D_f by the fractal equation (Sec. 3.1); the
 * box-counting D_f.  Pair distances and box indices are computed in float64.
 */
int npsim_stats(npsim_sim_t sim, const npsim_stats_cfg_t *cfg, int64_t *rdf_counts,
                double *rdf_g, int64_t *radial_counts, double *radial_c,
                npsim_stats_t *out);

/*
 * Light scattered by the NPs (Sec. 3.3): the intensity as the Fourier transform
 * of the RDF, I(q) = N_surf^2 * integral of exp(i q.r) g(r) d^3r, for g constant
 * on each of the n_bins bins of [0, r_max) (the g of npsim_stats):
 *   I(q) = N_surf^2 4 pi sum_b g_b [G(q r_{b+1}) - G(q r_b)] / q^3,
 *   G(u) = sin u - u cos u,  and  N_surf^2 4 pi sum_b g_b (r_{b+1}^3 - r_b^3)/3 at q = 0;
 * with I_frac (or NULL) also the fractal form I_frac(q) = N_surf^2 (q R_g)^(-D_f).
 * g (n_bins), q (n_q, >= 0), I and I_frac (n_q) are host arrays; the sums run on
 * the GPU in float64 (one warp per q, bins reduced in a fixed order).  Errors:
 * INVALID_ARG (NULL arrays, n_bins or n_q < 1, r_max <= 0, q < 0), CUDA.
 */
int npsim_scattering(const double *g, int32_t n_bins, double r_max, double n_surf, double Rg,
                     double Df, const double *q, int32_t n_q, double *I, double *I_frac);

/* Checkpoint (Sec. 2.2: a run can be halted and resumed from its saved NP
 * configuration, possibly with other parameters): the raw state words
 * (position hi and lo float32 words, float32 velocities), types, step counter,
 * parameters and the order in which the pair kernels sum over the NPs, so that
 * a resumed run is bit-identical to an uninterrupted one.  npsim_load creates a new object; params_override (or NULL) replaces
 * the saved scenario parameters, types_override likewise.  Errors: IO (file
 * cannot be opened, is truncated or is not a checkpoint of this format). */
int npsim_save(npsim_sim_t sim, const char *path);
int npsim_load(const char *path, const npsim_type_t *types_override,
               const npsim_params_t *params_override, void *stream, npsim_sim_t *out);

/* Test hook: n_blocks Philox4x32-10 blocks computed on the device, block b with
 * counter (ctr[0] + b (carry into ctr[1]), ctr[1], ctr[2], ctr[3]) and key
 * (seed low word, seed high word), copied to host out[4*n_blocks]. */
int npsim_philox(uint64_t seed, const uint32_t ctr[4], int64_t n_blocks, uint32_t *out);

/* Test hook: the three standard normals per particle that step `step` uses
 * (Box-Muller on Philox counter (i, step, 0)), n x 3 into host out. */
int npsim_normals(uint64_t seed, int64_t step, int64_t n, double *out);

/* Launch shape of the all-pairs kernel chosen by the autotuner: threads per
 * CTA, particles i per thread, j-tile length, CTAs launched, the index of the shape in
 * the autotuner's table, and 1 if it is the packed float32x2 Coulomb kernel, 2
 * if it is the packed Coulomb kernel over partners grouped by charge value, 3
 * if it is the packed LJ + Coulomb kernel over partners grouped by type (0: the
 * scalar kernel).  Any pointer may be NULL.  The grouped kernels (2, 3) cut
 * their work into a number of ranges per CTA that the autotuner also picks and
 * hand the ranges out at run time.  The environment variable
 * NPSIM_AUTOTUNE=1:<index>[:<ranges per CTA>] forces a shape at npsim_create
 * (NPSIM_AUTOTUNE=0: the first shape); with
 * NPSIM_AUTOTUNE_LOG set, the autotuners print every candidate's time to stderr. */
int npsim_allpairs_config(npsim_sim_t sim, int *block, int *i_per_thread, int *j_tile,
                          int *grid, int *index, int *packed);

/* Number of stream-K ranges the all-pairs work is cut into (each writes its
 * own partial slot; equal to the CTAs launched unless the shape is a grouped
 * one, whose CTAs take further ranges from a device counter as they finish);
 * 0 without an all-pairs sum. */
int npsim_allpairs_ranges(npsim_sim_t sim, int *ranges);

/* Number of launch shapes in the autotuner's table. */
int npsim_allpairs_num_configs(int *count);

/* ------------------------------------------------------------------------
 * Ensemble: many independent droplets (each the system of Sec. 2 with its own
 * types, charges, radius law and seed) advanced together.  One all-pairs launch
 * and one integrator launch per step cover every droplet: the (i-tile x
 * j-tile) work rectangles of all droplets are laid end to end and split evenly
 * over the CTAs, so droplets of very different N share the GPU in one launch.
 * Steps replay from captured CUDA graphs; the launch shape is chosen by timing
 * every candidate at npsim_ens_create (NPSIM_ENS_SHAPE=<index> forces one).
 */
typedef struct npsim_ens *npsim_ens_t;

/* One droplet: same meaning as the arguments of npsim_create.  params.lj_mode
 * must be 0 or 1 (the ensemble sums LJ inside the all-pairs kernel);
 * params.sum_neutral is ignored (the ensemble sums LJ and Coulomb in one pass). */
typedef struct {
    int64_t n;
    const npsim_type_t *types; /* params.n_types entries */
    npsim_params_t params;
    const double *x0;          /* n x 3 */
    const double *v0;          /* n x 3 or NULL (zero) */
    const int32_t *type;       /* n */
} npsim_droplet_t;

/* Create an ensemble of n_drops droplets (the library copies all inputs) and
 * compute the initial forces.  Errors as npsim_create, per droplet. */
int npsim_ens_create(const npsim_droplet_t *drops, int32_t n_drops, void *stream,
                     npsim_ens_t *out);

/* Advance every droplet by n_steps steps (all droplets share the step counter);
 * one device-to-host read of the error word at the end: NONFINITE or ESCAPED
 * (per droplet, as npsim_step). */
int npsim_ens_step(npsim_ens_t ens, int64_t n_steps);

/* State of droplet d (host arrays, any may be NULL; n_d x 3). */
int npsim_ens_get_state(npsim_ens_t ens, int32_t d, double *x, double *v, double *F,
                        int64_t *step);

/* Total forces of droplet d at the current state (recomputed), n_d x 3. */
int npsim_ens_forces(npsim_ens_t ens, int32_t d, double *F);

/* Statistics of Sec. 3 of droplet d at the ensemble's current step, computed on
 * the device from the ensemble's own state (no copy of the positions to the
 * host): the same outputs, definitions and units as npsim_stats -- the RDF of
 * Sec. 3.2 (ordered-pair counts and g, V the droplet's volume 4 pi R_d(t)^3 / 3),
 * the radial concentration C_NPs, N_surf, R_g and D_f by the fractal equation
 * (Sec. 3.1, Eqs. N, Rg, r0, with the droplet's number-mean diameter) and the
 * box-counting D_f.  Host outputs as in npsim_stats (rdf_counts/rdf_g n_bins,
 * radial_counts/radial_c radial_bins; any of the four may be NULL).  Scratch is
 * allocated on the first call and grown for larger droplets; the call
 * synchronises the ensemble's stream.  Errors: INVALID_ARG (d outside
 * [0, n_drops), bad cfg), OOM, CUDA. */
int npsim_ens_stats(npsim_ens_t ens, int32_t d, const npsim_stats_cfg_t *cfg,
                    int64_t *rdf_counts, double *rdf_g, int64_t *radial_counts,
                    double *radial_c, npsim_stats_t *out);

/* Launch shape of the ensemble all-pairs kernel (any pointer may be NULL). */
int npsim_ens_config(npsim_ens_t ens, int *block, int *i_per_thread, int *j_tile, int *grid,
                     int *index);

/* Total NPs and ordered pairs sum_d n_d (n_d - 1) per step. */
int npsim_ens_info(npsim_ens_t ens, int64_t *n_total, double *pairs_per_step);

/* Work items of one all-pairs launch (row tile x run of j-tiles, over all
 * droplets) and rows per tile (either pointer may be NULL): each item writes
 * one partial slot of 6 x itile floats that the integrator reads (measurement
 * hook: the integrator's bytes). */
int npsim_ens_work(npsim_ens_t ens, int64_t *n_items, int32_t *itile);

/*
 * Per-kernel timing of the ensemble (measurement hook).  enable = 1 re-captures
 * the step graphs with CUDA event records around the all-pairs launch and the
 * integrator launch of every step of a chunk; enable = 0 removes them (results
 * do not depend on it).  After an npsim_ens_step, npsim_ens_kernel_times writes
 * the mean duration in milliseconds of the all-pairs launch (ms[0]) and of the
 * integrator launch (ms[1]) over the steps of the last replayed graph chunk,
 * and the number of steps averaged.  ms must hold 2 doubles.  Errors:
 * INVALID_ARG (NULL ensemble or ms, profiling not enabled), CUDA.
 */
int npsim_ens_profile(npsim_ens_t ens, int enable);
int npsim_ens_kernel_times(npsim_ens_t ens, double *ms, int *samples);

void npsim_ens_destroy(npsim_ens_t ens);

/* ------------------------------------------------------------------------
 * Learned surrogate (no counterpart in the paper): a deep ensemble of n_nets
 * multilayer perceptrons, n_in inputs -> n_layers hidden layers of n_hidden
 * units with SiLU -> n_out outputs, mapping scenario parameters to statistics
 * of the final aggregate (fractal dimension, RDF bins).  BF16 weights and
 * activations, FP32 accumulation on the tcgen05 tensor cores, FP32 master
 * weights trained with AdamW by the library's own forward and backward
 * kernels.  Inputs and targets are standardised with npsim_surr_set_norm.
 * Host arrays are row-major float32 (samples x features).  The library owns the
 * object and its device memory; calls use the object's own stream and return
 * after synchronising it.
 */
typedef struct npsim_surr *npsim_surr_t;

/* Shape limits: n_in <= 64, n_hidden in [16, 256] step 16, 1..8 hidden layers,
 * n_out <= 256, 1..64 networks.  Weights: He-uniform from `seed`, biases 0. */
int npsim_surr_create(int32_t n_in, int32_t n_hidden, int32_t n_layers, int32_t n_out,
                      int32_t n_nets, uint64_t seed, npsim_surr_t *out);
void npsim_surr_destroy(npsim_surr_t s);

/* Standardisation x' = (x - x_mean) / x_std, y' = (y - y_mean) / y_std (NULL =
 * 0 mean / unit std).  Standard deviations must be positive. */
int npsim_surr_set_norm(npsim_surr_t s, const float *x_mean, const float *x_std,
                        const float *y_mean, const float *y_std);

/* Parameters of one network as a flat float32 vector: for each layer in order
 * W (out_pad x in_pad, row-major; in_pad = n_in or n_hidden rounded up to 16,
 * out_pad = n_hidden or n_out rounded up to 16) then b (out_pad).  Padded
 * entries are zero.  get also returns the last computed gradients (either
 * pointer may be NULL). */
int npsim_surr_param_count(npsim_surr_t s, int64_t *count);
int npsim_surr_get_params(npsim_surr_t s, int32_t net, float *flat, float *grads);
int npsim_surr_set_params(npsim_surr_t s, int32_t net, const float *flat);

/* Test hook: forward and backward pass of network `net` on B samples (X: B x n_in,
 * Y: B x n_out, raw units), no update.  Mean-squared error over the
 * standardised outputs; gradients in the flat layout (param_count floats);
 * loss and the standardised prediction Yhat (B x n_out) optional. */
int npsim_surr_grads(npsim_surr_t s, int32_t net, const float *X, const float *Y, int32_t B,
                     float *grads, float *loss, float *Yhat);

/* Train every network of the ensemble for `epochs` passes over n_samples samples
 * with AdamW (beta 0.9 / 0.999, eps 1e-8, decoupled weight decay wd on weights),
 * minibatches of `batch`, each network with its own shuffled order.  final_loss
 * (optional): loss of the last minibatch. */
int npsim_surr_train(npsim_surr_t s, const float *X, const float *Y, int32_t n_samples,
                     int32_t epochs, int32_t batch, float lr, float wd, uint64_t shuffle_seed,
                     float *final_loss);

/* Predict B samples: mean over the networks (B x n_out, raw units) and the
 * spread, the standard deviation across networks (B x n_out, may be NULL). */
int npsim_surr_predict(npsim_surr_t s, const float *X, int32_t B, float *Y_mean,
                       float *Y_spread);

/* Test hook: C = A B^T on the tcgen05 GEMM kernel for host BF16 matrices (bit
 * patterns; A: M x K, B: N x K, row-major), C: M x N float32.  N, K and n_tile
 * must be multiples of 16, n_tile <= 256. */
int npsim_gemm_bf16(const uint16_t *A, const uint16_t *B, int32_t M, int32_t N, int32_t K,
                    int32_t n_tile, float *C);

/* Test hook of the failure path of the tensor-core kernels (no counterpart in the
 * paper): every mbarrier wait of the GEMM kernel's main loop (TMA operand ring,
 * MMA pipeline, accumulator ready) gives up after `cycles` SM clock cycles
 * instead of the default 2^32 (~2 s), for every GEMM launched after the call
 * from any thread (the surrogate's training and gradient passes and
 * npsim_gemm_bf16); 0 restores the default.  A wait that gives up makes the
 * kernel set its error flag, wait with the default bound for its copies and
 * MMAs in flight, free its tensor memory and return without writing its
 * output; the call that launched it returns NPSIM_ERR_TIMEOUT.  This lets a
 * test drive that path without a stuck GPU.  Errors: INVALID_ARG (cycles < 0). */
int npsim_test_wait_cycles(int64_t cycles);

/*
 * All-pairs Coulomb forces without any device allocation.  The paper has no
 * counterpart: this entry point serves callers that cannot call cudaMalloc when
 * they need forces -- code running under a framework whose own memory pool owns
 * all device memory and forbids raw allocations, or a real-time loop that cannot
 * risk an allocation's latency or its failure in the middle of a run.
 *
 * Computes F_i = C q_i sum_{j != i} q_j (x_i - x_j) / |x_i - x_j|^3, the same sum
 * as npsim_forces(sim, 3, ...), from dev_xyzq (device, n float4 records
 * (x, y, z, q) in float32, e.g. filled by npsim_positions_device) into dev_F
 * (device, n x 3 float64, row-major).  Both buffers are the caller's.  C is
 * `bjerrum`.  Work is queued on `stream`; the call does not synchronise.
 *
 * Scratch: the partial sums live in one fixed __device__ array of 3.75 MiB that
 * every GPU loading the library holds until the process exits.  n must be in
 * [1, 32768]; larger n is rejected with NPSIM_ERR_INVALID_ARG.  The first call
 * on a device looks up the array's device address for that device (set-up,
 * once per device, with that device current); make that first call before any
 * stream capture.  The address is kept while the calling thread's current
 * context stays the one the set-up ran in, and looked up again when it changes
 * (after a cudaDeviceReset, for instance, the array lives at a new address in
 * the new context).  Every call on a device shares the array: calls that
 * overlap on the GPU (different streams without ordering) race and give wrong
 * forces.  Each
 * call writes every partial it reads, so nothing carries over from the previous
 * call.  Allocates nothing (no cudaMalloc/cudaFree).
 */
int npsim_coulomb_forces_noalloc(const float *dev_xyzq, int64_t n, double bjerrum,
                                 double *dev_F, void *stream);

/*
 * Measurement hook: the FP32 CUDA-core rate that bounds the all-pairs kernels
 * (their pair body is FP32 arithmetic, not a dense contraction).  One launch of
 * one full wave of CTAs (every SM filled to its occupancy limit), each thread
 * running 8 independent chains of `iters` dependent fused multiply-adds:
 * scalar FFMA (packed = 0, 2 flops per lane) or the packed float32x2 FFMA2 the
 * pair kernels issue (packed = 1, 4 flops per lane), after one shorter warm-up
 * launch, timed with CUDA events on `stream`.  *flops: floating-point
 * operations of the timed launch; *ms: its duration; *grid (may be NULL): CTAs
 * launched.  The achieved rate is *flops / *ms; it depends on the SM clock
 * during the launch, which the caller samples.  Allocates a small sink buffer;
 * synchronises the stream.  Errors: INVALID_ARG (iters outside [1, 2^40],
 * NULL outputs), CUDA, NO_DEVICE. */
int npsim_fma_peak(int packed, int64_t iters, void *stream, double *flops, float *ms,
                   int *grid);

/* Kernel launches per step in a long run (pair kernels + cell-list kernels + one
 * integrator pass); npsim_step adds one integrator launch per graph chunk. */
int npsim_launches_per_step(npsim_sim_t sim, int *launches);

/* Cell grid of the LJ cell list (lj_mode 2): cells per axis and in total; both
 * 0 when the scenario has no cell list.  The grid covers [-L, L)^3 with L the
 * largest |coordinate| at creation (or R0) plus the largest cutoff, cell edge
 * >= the largest cutoff. */
int npsim_cell_grid(npsim_sim_t sim, int *dim, int64_t *n_cells);

/* Verlet neighbour lists of the cell-list LJ (lj_mode 2): the list capacity per
 * NP, the mean list length at the last build, and the number of builds run so
 * far (a build runs when an NP has moved more than half the skin since the
 * previous one).  All 0 without a cell list. */
int npsim_nbr_info(npsim_sim_t sim, int *cap, double *mean_len, int64_t *builds);

/* Steps per captured CUDA graph (npsim_step replays ceil(n / chunk) graphs). */
int npsim_chunk_steps(npsim_sim_t sim, int *chunk);

/*
 * Per-kernel timing.  enable = 1 re-captures the step graphs with CUDA event
 * records around the kernels of every step (all-pairs forces, cell-list
 * build, cell-list LJ, integrator); enable = 0 removes them.  After an
 * npsim_step, npsim_kernel_times writes the mean duration in milliseconds of
 * each of the four groups over the steps of the last replayed graph chunk
 * (0 for groups this scenario does not launch) and the number of steps
 * averaged.  ms must hold 4 doubles.
 */
int npsim_profile(npsim_sim_t sim, int enable);
int npsim_kernel_times(npsim_sim_t sim, double *ms, int *samples);

#ifdef __cplusplus
}
#endif

#endif /* NPSIM_H */
