/*
 * jwf.h -- C ABI of libjwf, a GB300 (sm_103a) engine for the stochastic
 * cellular-automaton wildfire model of JaxWildfire (arXiv 2512.06102).
 *
 * One context (jwf_ctx) holds a batch of N independent grids ("envs"), each
 * with its own height H[e] and width W[e] (ragged batches are allowed).  The
 * context owns the device state, the per-(cell, direction) probability and
 * rate tables and the per-env counters; callers own every pointer they pass.
 *
 * Conventions shared by every entry point
 *  - Cells of env e occupy the contiguous index range [off[e], off[e] + H*W),
 *    row-major (x fastest), off[e] = sum of the sizes of envs before e.
 *    "cells" below is the total over all envs.
 *  - Cell states (uint8): 0 no fuel (an unburned cell whose fuel density
 *    mu_den is -1; it can never ignite), 1 can burn, 2 burning, 3 burned
 *    (Section 3, "State representation": F in {unburned, burning, burned}).
 *  - Directions d = 0..7 (east, north-east, north, north-west, west,
 *    south-west, south, south-east): the angle of Delta_d is d*45 degrees,
 *    east = 0, counter-clockwise (Section 3, below Eq. 2).  Rows grow
 *    southward, so north is row - 1.  Tables are indexed [cell v][d] and
 *    describe spread INTO target v FROM source u = v - Delta_d.
 *  - Pointers named d_* are device pointers (cudaMalloc / torch tensors),
 *    h_* are host pointers.  Every call is asynchronous on the given
 *    cudaStream_t (passed as void*; NULL = the legacy default stream) and
 *    returns once the work is enqueued.  Argument errors are reported
 *    immediately and leave the context unchanged.  An error raised inside a
 *    kernel (a bounded wait that ran out: the tiled step's wait for its
 *    tensor copy) is written to a device status word and reported by
 *    jwf_sync().
 *  - No call aborts, throws or traps; every failure is a jwf_status.
 *  - One context must be used from one stream at a time (calls on one
 *    context that overlap on the GPU race).
 */
#ifndef JWF_H
#define JWF_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define JWF_API __attribute__((visibility("default")))
#else
#define JWF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct jwf_ctx jwf_ctx;

typedef enum {
    JWF_OK = 0,
    JWF_EINVAL = 1,        /* bad argument (null pointer, size, range)        */
    JWF_ENOMEM = 2,        /* device or host allocation failed                */
    JWF_ECUDA = 3,         /* a CUDA runtime call failed (see jwf_last_error) */
    JWF_ETIMEOUT = 4,      /* a bounded device-side wait gave up              */
    JWF_ESTATE = 5,        /* call out of order (e.g. step before load_state) */
    JWF_EUNSUPPORTED = 6   /* option not available for this configuration     */
} jwf_status;

/* Flags of jwf_config.flags */
#define JWF_AUTO_RESET     0x1u  /* a done env restarts from its initial state  */
#define JWF_WIND_PER_CELL  0x2u  /* wind arrays are [cells], not [n_envs]       */
#define JWF_KEEP_RATES     0x4u  /* keep the rate table r (relaxed path)        */

typedef struct {
    int32_t n_envs;          /* N >= 1                                           */
    const int32_t* h_H;      /* [N] grid heights, 1..65535 (copied)              */
    const int32_t* h_W;      /* [N] grid widths, 1..65535 (copied)               */
    int32_t n_classes;       /* landcover classes, 1..16                         */
    uint64_t seed;           /* Philox key (low word, high word)                 */
    int32_t t_max;           /* episode length limit; <= 0: none                 */
    int32_t drop_radius;     /* tanker drop: (2R+1)^2 square, R >= 0 (1 = 3x3)   */
    uint32_t flags;          /* JWF_* flags above                                */
} jwf_config;

/* Model parameters (Section 3, Eqs. 1-4 and the stochastic update). */
typedef struct {
    float p_base;            /* base propagation factor, Eq. 3                   */
    float alpha_w1;          /* wind-speed coefficient, Eq. 1                    */
    float alpha_w2;          /* wind-direction coefficient, Eq. 1                */
    float alpha_s;           /* slope coefficient per degree, Eq. 2              */
    float alpha_gamma;       /* susceptibility scale, gamma(v), Section 3        */
    float p_continue;        /* probability that a burning cell keeps burning    */
    float cell_size;         /* metres per cell (slope run length)               */
    const float* h_mu_veg;   /* [n_classes] canopy modifiers in [-1, 1] (copied) */
    const float* h_mu_den;   /* [n_classes] fuel density in [-1, 1]; -1 = none   */
} jwf_params;

/* Number of doubles in a parameter-gradient vector:
 * [p_base, alpha_w1, alpha_w2, alpha_s, alpha_gamma, mu_veg[C], mu_den[C]] */
#define JWF_GRAD_SIZE(n_classes) (5 + 2 * (n_classes))

/* ---- lifetime ------------------------------------------------------------ */

/* Create a context for cfg (host struct, read during the call).  Allocates the
 * state, the probability table, the per-env counters and, with
 * JWF_KEEP_RATES, the rate table on the current CUDA device.  *out is NULL on
 * failure.  Errors: JWF_EINVAL (bad sizes or flags), JWF_ENOMEM, JWF_ECUDA. */
JWF_API jwf_status jwf_create(const jwf_config* cfg, jwf_ctx** out);

/* Release everything the context owns.  Waits for the device.  NULL is a no-op. */
JWF_API jwf_status jwf_destroy(jwf_ctx* ctx);

/* Store the parameters used by later calls (copied; mu tables are host arrays
 * of n_classes floats).  Errors: JWF_EINVAL (NULL, p_continue outside [0,1],
 * mu outside [-1,1], negative coefficients where the paper requires >= 0). */
JWF_API jwf_status jwf_set_params(jwf_ctx* ctx, const jwf_params* p);

/* Block until the stream's work is done, then report (and clear) any error a
 * kernel recorded in the device status word. */
JWF_API jwf_status jwf_sync(jwf_ctx* ctx, void* stream);

JWF_API const char* jwf_status_string(jwf_status s);
JWF_API const char* jwf_last_error(const jwf_ctx* ctx);   /* message of the last failure */

/* Read-only facts about the context. */
JWF_API int32_t jwf_n_envs(const jwf_ctx* ctx);
JWF_API int64_t jwf_n_cells(const jwf_ctx* ctx);
JWF_API int64_t jwf_env_offset(const jwf_ctx* ctx, int32_t e);     /* off[e]; e == N gives cells */

/* ---- probability tables (Section 3, Eqs. 1-4) ---------------------------- */

/* Build the per-(cell, direction) tables on the device from landcover class
 * ids (uint8 [cells], < n_classes), elevation (float [cells], metres) and
 * wind speed (m/s, >= 0) and direction (radians; the direction the wind
 * blows toward) given per env ([N]) or, with JWF_WIND_PER_CELL, per cell.
 * For target v, direction d, source u = v - Delta_d:
 *   S(u,d)   = atan((z(v) - z(u)) / (cell_size * |Delta_d|)) in degrees (Eq. 2)
 *   phi(u,d) = p_base (1 + mu_veg(u)) (1 + mu_den(u))
 *              exp(alpha_w1 V(u)) exp(alpha_w2 V(u) (cos(d*pi/4 - Theta(u)) - 1))
 *              exp(alpha_s S(u,d))                                   (Eqs. 1-3)
 *   gamma(v) = alpha_gamma (1 + mu_veg(v)) (1 + mu_den(v))           (Section 3)
 *   r[v][d]  = gamma(v) phi(u,d), 0 when u is outside the grid       (Eq. 4 rate)
 *   q[v][d]  = 1 - exp(-r[v][d]), the probability that a burning u ignites v
 *              in one step; over all burning neighbours this gives exactly
 *              Eq. 4's 1 - exp(-gamma(v) * lambda).
 * Uses the parameters of the last jwf_set_params().  Writes q (and r with
 * JWF_KEEP_RATES).  Errors: JWF_ESTATE (no parameters), JWF_EINVAL (NULL). */
JWF_API jwf_status jwf_precompute_probs(jwf_ctx* ctx, const uint8_t* d_class, const float* d_dem,
                                const float* d_wind_speed, const float* d_wind_dir, void* stream);

/* Register the terrain the fused step kernel (JWF_KERNEL_FUSED) evaluates
 * Eqs. 1-4 from, without building the table: landcover class ids (uint8
 * [cells]), elevation (float [cells]) and per-env wind speed and direction
 * (float [N]; per-cell wind is JWF_EUNSUPPORTED here).  The pointers are
 * borrowed: the caller keeps the buffers alive and unchanged while it steps.
 * jwf_precompute_probs registers its inputs the same way.  Uses the
 * parameters of the last jwf_set_params (later parameter changes are picked
 * up by the next jwf_step). */
JWF_API jwf_status jwf_set_terrain(jwf_ctx* ctx, const uint8_t* d_class, const float* d_dem,
                                   const float* d_wind_speed, const float* d_wind_dir, void* stream);

/* Wind as a time series (Section 3 indexes wind speed and direction by the
 * step; Section 4 lets weather change over a run).  d_wind_speed and
 * d_wind_dir are float [n_steps][N] on the device, borrowed (they must stay
 * valid while the series is set: the wind part of Eqs. 1-2 is recomputed from
 * them when the parameters change).  A step of an env at episode step t uses
 * row min(t, n_steps - 1), so the series restarts with every episode.  Only
 * the fused kernels (JWF_KERNEL_FUSED, JWF_KERNEL_TILED_FUSED, and AUTO with
 * terrain set) evaluate rates per step; jwf_step with a table kernel returns
 * JWF_EUNSUPPORTED while a series is set.  n_steps = 0 returns to the static
 * wind of jwf_set_terrain.  Allocates device memory when the series grows. */
JWF_API jwf_status jwf_set_wind_series(jwf_ctx* ctx, int32_t n_steps, const float* d_wind_speed,
                                       const float* d_wind_dir, void* stream);

/* Replace the tables with caller data: d_q float [cells][8] (required),
 * d_r float [cells][8] (may be NULL; requires JWF_KEEP_RATES otherwise).
 * Device-to-device copies on the stream. */
JWF_API jwf_status jwf_set_probs(jwf_ctx* ctx, const float* d_q, const float* d_r, void* stream);

/* Borrowed device views of the tables (valid until jwf_destroy). */
JWF_API jwf_status jwf_get_probs(jwf_ctx* ctx, float** d_q, float** d_r);

/* Diagnostics of the fused step kernels' ignition test (Section 3
 * "Stochastic update", Eqs. 1-4).  Those kernels compare a pair's draw u with
 * a plain-float probability p_f and a bound B on |p_f - p|, p the probability
 * jwf_precompute_probs writes; only a draw within B of p_f takes the exact
 * double-float rate, so the outcome is always u < p.  For n tuples (target
 * class d_class_v[i], source class d_class_u[i], elevations d_z_v[i] and
 * d_z_u[i] in m, the wind part of the exponent at the source as hi + lo in
 * d_wexp[2i], d_wexp[2i + 1], direction d_dir[i] in 0..7 as in jwf_step) and
 * the context's parameters, writes d_out[3i .. 3i + 2] = p_f, B, p (float).
 * All pointers are device memory of n (d_wexp 2n, d_out 3n) elements, read or
 * written on the stream.  Errors: JWF_ESTATE (no parameters), JWF_EINVAL (null
 * pointer with n > 0, n < 0). */
JWF_API jwf_status jwf_check_prob_bound(const jwf_ctx* ctx, int64_t n, const uint8_t* d_class_v,
                                        const uint8_t* d_class_u, const float* d_z_v, const float* d_z_u,
                                        const float* d_wexp, const int32_t* d_dir, float* d_out, void* stream);

/* ---- discrete (stochastic) simulation (Section 3, "Stochastic update") --- */

/* Start a run: the initial states d_F0 (uint8 [cells], values 0..3) are
 * copied into the context as both the current state and the restart state of
 * every env; t = 0 and episode = 0 for all envs. */
JWF_API jwf_status jwf_load_state(jwf_ctx* ctx, const uint8_t* d_F0, void* stream);

/* 2-bit packed states.  A state 0..3 takes two bits: cell i of an array
 * (for the context, the cells of all envs in order, row-major within an
 * env) sits in bits 2(i mod 4) and 2(i mod 4) + 1 of byte i / 4, so a packed
 * array of n states takes ceil(n / 4) bytes, a quarter of the byte-per-cell
 * layout (the host-to-device copy of a batch's initial fires, a recorded
 * trajectory).  jwf_packed_size(n) is ceil(n / 4) rounded up to a multiple of
 * 16: the row stride of a packed history and the size to allocate. */
JWF_API int64_t jwf_packed_size(int64_t n_cells);

/* Pack n uint8 states (device, only their low two bits are kept) into
 * d_packed (device, ceil(n / 4) bytes written), or unpack them back.
 * Buffers are caller-owned and must not overlap.  Asynchronous on stream.
 * Errors: JWF_EINVAL (n < 0, null pointer with n > 0), JWF_ECUDA. */
JWF_API jwf_status jwf_pack_states(int64_t n_cells, const uint8_t* d_states, uint8_t* d_packed, void* stream);
JWF_API jwf_status jwf_unpack_states(int64_t n_cells, const uint8_t* d_packed, uint8_t* d_states, void* stream);

/* jwf_load_state from 2-bit packed initial states (device, ceil(cells / 4)
 * bytes).  The context keeps one byte a cell internally. */
JWF_API jwf_status jwf_load_state_packed(jwf_ctx* ctx, const uint8_t* d_P0, void* stream);

/* The current state of every env, 2-bit packed into d_packed (device,
 * caller-owned, ceil(cells / 4) bytes).  Errors: JWF_ESTATE (no state). */
JWF_API jwf_status jwf_get_state_packed(jwf_ctx* ctx, uint8_t* d_packed, void* stream);

/* Restart the envs selected by d_env_mask (uint8 [N], nonzero = restart; NULL
 * = all): state := initial state, t := 0, episode += 1 (a fresh random
 * stream).  Section 4: episodes restart from randomised initial fires. */
JWF_API jwf_status jwf_reset(jwf_ctx* ctx, const uint8_t* d_env_mask, void* stream);

/* Air-tanker action (Section 4: water turns a burning cell into a burned
 * one): every burning cell with d_mask[cell] != 0 (uint8 [cells]) becomes
 * burned.  Other cells are untouched. */
JWF_API jwf_status jwf_apply_action(jwf_ctx* ctx, const uint8_t* d_mask, void* stream);

/* Advance every env by k >= 1 synchronous steps.  Step s of env e:
 *   1. action: if d_drops is not NULL, d_drops[(s*N + e)*2 + {0,1}] is the
 *      (column, row) centre of a square drop of radius drop_radius (clipped
 *      to the grid; a negative centre means no drop); burning cells under it
 *      become burned;
 *   2. spread: every can-burn cell v with a burning neighbour u = v - Delta_d
 *      ignites if any such u succeeds its draw U(v,d) < q[v][d]; every burning
 *      cell stays burning if U(v) < p_continue, otherwise becomes burned
 *      (all draws from the post-action state, all cells at once);
 *   3. counts of burning and burned cells after the step go to
 *      d_burning[s*N + e], d_burnt[s*N + e] (int32 [k][N], may be NULL);
 *      done = (no burning cell) or (t >= t_max) goes to d_done[s*N + e]
 *      (uint8 [k][N], may be NULL); with JWF_AUTO_RESET a done env restarts
 *      (its reported counts are the pre-restart ones).
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11), key = seed, counter
 * = (y*W + x, t, env, 4*episode + slot); slot 0 -> directions 0..3, slot 1
 * -> directions 4..7, slot 2 word 0 -> the remain-burning draw; uniform =
 * (word >> 8) * 2^-24.  Results do not depend on the kernel chosen.
 * Errors: JWF_ESTATE (no table or no state loaded), JWF_EINVAL (k < 1). */
JWF_API jwf_status jwf_step(jwf_ctx* ctx, int32_t k, const int32_t* d_drops, int32_t* d_burning,
                    int32_t* d_burnt, uint8_t* d_done, void* stream);

/* Tanker actions as cell masks (Section 4: water turns a burning cell into a
 * burned one; any footprint, not only square drops).  A mask travels as a bit
 * row of jwf_mask_words(n_cells) uint32 words: cell g of the context (the
 * concatenated envs) at bit g % 32 of word g / 32, set = water on the cell.
 * jwf_pack_masks turns uint8 masks [n_rows][n_cells] (device, nonzero =
 * water) into n_rows such rows at d_bits (device, caller-owned,
 * n_rows * jwf_mask_words(n_cells) words); JWF_EINVAL for negative sizes or
 * null pointers with n_rows, n_cells > 0. */
JWF_API int64_t jwf_mask_words(int64_t n_cells);
JWF_API jwf_status jwf_pack_masks(int32_t n_rows, int64_t n_cells, const uint8_t* d_masks, uint32_t* d_bits,
                                  void* stream);

/* jwf_step with the action of step s given by mask row s of d_mask_bits
 * (uint32 [k][jwf_mask_words(cells)], device, read-only): step 1 of every env
 * turns its burning cells with a set bit into burned ones, then the spread
 * and the counts are those of jwf_step.  Every step kernel (resident, tiled,
 * plain) takes the masks inside its k-step launches.  Errors as jwf_step;
 * JWF_EINVAL when d_mask_bits is NULL. */
JWF_API jwf_status jwf_step_masked(jwf_ctx* ctx, int32_t k, const uint32_t* d_mask_bits, int32_t* d_burning,
                                   int32_t* d_burnt, uint8_t* d_done, void* stream);

/* jwf_step that also records the state after every step: d_history is uint8
 * [k][cells] on the device (row s = the state after step s, after an
 * auto-reset the restarted state; caller-owned).  The trajectory is the one
 * jwf_step produces.  The tiled kernels run one step per launch while
 * recording.  Errors as jwf_step; JWF_EINVAL when d_history is NULL. */
JWF_API jwf_status jwf_step_record(jwf_ctx* ctx, int32_t k, const int32_t* d_drops, int32_t* d_burning,
                                   int32_t* d_burnt, uint8_t* d_done, uint8_t* d_history, void* stream);

/* jwf_step_record with 2-bit packed rows: d_history is [k] rows of
 * jwf_packed_size(cells) bytes (device, caller-owned), row s = the packed
 * state after step s; a quarter of the memory of the byte-per-cell history
 * (e.g. 200 steps of 4096 grids of 128 x 128: 3.4 GB instead of 13.4 GB).
 * The resident kernels write the rows from their bit planes; the others pack
 * the state after each step.  Errors as jwf_step_record. */
JWF_API jwf_status jwf_step_record_packed(jwf_ctx* ctx, int32_t k, const int32_t* d_drops, int32_t* d_burning,
                                          int32_t* d_burnt, uint8_t* d_done, uint8_t* d_history, void* stream);

/* Replace the Philox key (the seed of jwf_create) for the following steps,
 * e.g. to draw a new sample of the same episode. */
JWF_API jwf_status jwf_set_seed(jwf_ctx* ctx, uint64_t seed);

/* Discrete states (uint8 [n][cells]) to relaxed planes (float [n][cells]
 * each): p_un = 1 for no-fuel and can-burn cells, p_burn = 1 for burning
 * cells, 0 otherwise (p_bd = 1 for burned cells is implicit).  With these
 * planes one relaxed step (Eqs. 5-10) is the expectation of the stochastic
 * step from the same state, which makes them the linearisation points of a
 * straight-through backward along a sampled trajectory. */
JWF_API jwf_status jwf_state_planes(jwf_ctx* ctx, int32_t n, const uint8_t* d_states, float* d_pun,
                                    float* d_pburn, void* stream);

/* Kernel choice for jwf_step (default JWF_KERNEL_AUTO: resident when every
 * env fits shared memory, else tiled, else (auto-reset) plain).  All kernels
 * give identical results for the same probabilities. */
typedef enum {
    JWF_KERNEL_AUTO = 0,      /* resident when every env fits shared memory  */
    JWF_KERNEL_PLAIN = 1,     /* one launch per step, state in global memory */
    JWF_KERNEL_RESIDENT = 2,  /* whole env in shared memory, k steps/launch  */
    JWF_KERNEL_FUSED = 3,     /* resident, evaluating the probability of each
                                 compared (target, source) pair from the
                                 terrain of jwf_set_terrain instead of reading
                                 the table; bit-identical to the table built
                                 by jwf_precompute_probs from that terrain;
                                 tiled (below) for envs too large for shared
                                 memory                                      */
    JWF_KERNEL_TILED = 4,     /* 128 x 256-cell tiles with a halo, up to 16
                                 steps per launch (temporal blocking); tiles
                                 with no fire within reach are skipped; for
                                 grids larger than shared memory.  Without
                                 JWF_AUTO_RESET only                          */
    JWF_KERNEL_TILED_FUSED = 5 /* tiled, probabilities from the terrain      */
} jwf_kernel;
/* Choose the step kernel; threads_per_env = 0 picks a block size by env size
 * (resident kernels) or 256 threads a tile (tiled kernels); else 32, 64, 128,
 * 256, 512 or 1024 threads per env (resident kernels) or 128, 256 or 512
 * threads a tile (tiled kernels).  Other values return JWF_EINVAL. */
JWF_API jwf_status jwf_set_kernel(jwf_ctx* ctx, jwf_kernel kernel, int32_t threads_per_env);

/* Resident envs run as up to four size classes by their longer side (<= 64,
 * <= 128, <= 256, > 256: classes 0..3), one persistent launch each, side by
 * side on forked streams.  jwf_size_classes writes the classes present to
 * h_classes (host, up to 4 entries, may be NULL) and returns their number;
 * jwf_set_class_threads sets the block size of one class (0: by size; 32,
 * 64, 128, 256, 512 or 1024), e.g. from an autotuner; a block size whose
 * shared memory (it grows with the warps) does not fit the class's largest env
 * returns JWF_EINVAL and changes nothing.  jwf_set_kernel's explicit
 * threads_per_env overrides both. */
JWF_API int32_t jwf_size_classes(const jwf_ctx* ctx, int32_t* h_classes);
JWF_API jwf_status jwf_set_class_threads(jwf_ctx* ctx, int32_t size_class, int32_t threads);

/* Steps per launch of the tiled kernel (1..16, default 16; the halo, and so
 * the redundant work per tile, grows with it). */
JWF_API jwf_status jwf_set_round_steps(jwf_ctx* ctx, int32_t steps);

/* How the tiled kernels stage a tile's region: 1 = one TMA tensor copy
 * (cp.async.bulk.tensor, the default where available), 0 = 128-bit loads by
 * all threads.  TMA serves the envs whose first cell and row pitch (W) are
 * multiples of 16 bytes; the others always take the loads.  Results do not
 * depend on the mode.  Errors: JWF_EINVAL (mode), JWF_EUNSUPPORTED (1 asked,
 * no env qualifies or the driver has no tensor-map encoder).
 * jwf_tile_copy returns the mode in effect. */
JWF_API jwf_status jwf_set_tile_copy(jwf_ctx* ctx, int32_t tma);
JWF_API int32_t jwf_tile_copy(const jwf_ctx* ctx);

/* Bound of the tiled kernels' wait for a tensor copy (default 2 s; 1 ns ..
 * 10 s).  A wait that runs out sets a bit of the device status word (the
 * tile is left unstepped) and jwf_sync returns JWF_ETIMEOUT.  With no_copy
 * != 0 (diagnostics only) the kernels arm the wait but issue no copy, so
 * every wait runs out: this exercises the timeout path without a fault. */
JWF_API jwf_status jwf_set_tile_copy_wait(jwf_ctx* ctx, uint64_t timeout_ns, int32_t no_copy);

/* Split a resident jwf_step of k >= 2 * steps steps into two launches: the
 * first `steps` steps in the queue order, then the rest with each size
 * class's envs reordered by their burning-cell count after the first part,
 * largest first (the envs with the longest fires then start first instead
 * of last).  Default 12; 0 never splits.  Applied to batches of one size
 * class (see jwf_size_classes) and not while recording a history.  Results
 * do not depend on it.  Errors: JWF_EINVAL (< 0). */
JWF_API jwf_status jwf_set_reorder_steps(jwf_ctx* ctx, int32_t steps);

/* Scheduling hint for the resident kernels: within each size class, envs are
 * taken from the work queue in descending h_priority (host float [N], read
 * during the call; e.g. the expected number of steps an env's fire lasts) so
 * that long envs start first and do not finish last.  NULL restores the
 * default order (cells descending).  Results do not depend on the order.
 * Synchronous (waits for work already queued on the device). */
JWF_API jwf_status jwf_set_env_priority(jwf_ctx* ctx, const float* h_priority);

/* Instrumentation: while d_counts (four uint64 on the device, owned by the
 * caller) is set, the resident step kernels add to them the work they did:
 * [0] (target, burning source) pairs compared (the table reads of the byte
 * model), [1] Philox blocks drawn for can-burn cells, [2] remain-burning
 * draws, [3] 32-cell bit-plane words scanned (one per word per step).
 * NULL switches counting off (the default). */
JWF_API jwf_status jwf_set_pair_counter(jwf_ctx* ctx, unsigned long long* d_counts);

/* Borrowed device views: current state uint8 [cells] and int32 [N] step
 * counters t and episode numbers (valid until the next call on ctx). */
JWF_API jwf_status jwf_get_state(jwf_ctx* ctx, uint8_t** d_state, int32_t** d_t, int32_t** d_episode);

/* ---- air-tanker agent environment (Section 4) ---------------------------- */

/* An agent per env moves over the grid and controls a valve that drops a
 * limited amount of water (water turns burning cells into burned cells);
 * it observes an egocentric window of the fire state; each step is penalised
 * per burning cell and an extinguished fire earns +10.  The paper states
 * these ingredients, not their details; this library's readings:
 *   d_agent: int32 [N][3] = (x, y, water) per env, device, caller-owned;
 *   action a in [0, 10): move = a % 5 (0 stay, 1 north = row - 1, 2 east =
 *     column + 1, 3 south, 4 west; clamped to the grid); the valve is open
 *     when a >= 5; other values count as 0;
 *   an open valve with water > 0 drops water on the drop footprint (radius
 *     drop_radius of jwf_config) centred on the agent's new cell and uses
 *     one unit; the drop is this step's action (applied before the spread);
 *   reward = -burn_penalty * (burning cells after the step) + (10 if none);
 *   observation: uint8 [N][obs_k][obs_k] (obs_k odd, <= 63), the states
 *     centred on the agent, 255 outside the grid (d_obs may be NULL);
 *   restart (jwf_agent_reset, and after a step that an auto-reset context
 *     restarted): Philox4x32-10 with the context's key and counter (0, 0,
 *     env, 4 * episode + 3): x = floor(u(w0) * W), y = floor(u(w1) * H),
 *     water = water0; with random_fire the first can-burn cell at or after
 *     cell floor(u(w2) * H * W) (row-major, wrapping) starts burning.
 * jwf_agent_step = move/valve, one jwf_step (k = 1, any kernel; use
 * JWF_AUTO_RESET for continuing episodes), reward, restarts, observation
 * (when every grid is at most 32 x 32 and the kernel is AUTO, RESIDENT or
 * FUSED, all of it in one launch with one warp per grid; same results);
 * d_actions int32 [N], d_reward float [N] and d_done uint8 [N] (both may be
 * NULL).  Errors: JWF_EINVAL for null d_agent/d_actions, water0 < 0 or a bad
 * obs_k; otherwise as jwf_step. */
JWF_API jwf_status jwf_agent_reset(jwf_ctx* ctx, int32_t* d_agent, int32_t water0, int32_t random_fire,
                                   int32_t obs_k, uint8_t* d_obs, void* stream);
JWF_API jwf_status jwf_agent_step(jwf_ctx* ctx, const int32_t* d_actions, int32_t* d_agent, int32_t water0,
                                  int32_t random_fire, float burn_penalty, float* d_reward, uint8_t* d_done,
                                  int32_t obs_k, uint8_t* d_obs, void* stream);

/* ---- relaxed (raw-probabilities) update, Eqs. 5-10 ----------------------- */

/* Kernels of the relaxed step.  JWF_RELAXED_TILED (default): the forward
 * walks 16 x 64-cell tiles staged in shared memory by asynchronous copies
 * (persistent CTAs, two tiles deep); the adjoint is one kernel in which each
 * warp sweeps a strip of 30 columns down the rows (a halo column on each
 * side), keeping the p_burn window, lam, glam and the per-source
 * accumulators of dL/dp_burn in registers and streaming its rows through a
 * shared-memory ring filled by asynchronous copies.  JWF_RELAXED_PLAIN: one
 * thread per cell; the adjoint is two kernels (lam adjoint, then the
 * transpose gather) with a round trip of glam through memory.  lam is summed
 * in the same order by both; the gather's order differs (rounding only).
 * Rates whose source lies outside the grid are multiplied by zero (they must
 * be finite; jwf_precompute_probs writes 0 there). */
enum jwf_relaxed_kernel { JWF_RELAXED_TILED = 0, JWF_RELAXED_PLAIN = 1 };
JWF_API jwf_status jwf_set_relaxed_kernel(jwf_ctx* ctx, int32_t kernel);

/* One deterministic step on probability planes (float [cells] each; p_bd =
 * 1 - p_un - p_burn is implicit).  With m = d_mask[cell] in [0,1] (float
 * [cells], NULL = 0) the tanker acts first: pb = (1 - m) p_burn.  Then
 *   lam(v)  = sum_d pb(v - Delta_d) r[v][d]        (gamma(v) lambda, Eq. 4
 *                                                  with b(u) := p_burn(u))
 *   p_ign   = 1 - exp(-lam)                        (Eq. 4)
 *   newly   = p_un p_ign                           (Eq. 5)
 *   p_un'   = p_un - newly                         (Eq. 9)
 *   p_burn' = newly + p_continue pb                (Eqs. 6, 8)
 * Requires JWF_KEEP_RATES and a rate table.  Outputs must not alias inputs. */
JWF_API jwf_status jwf_step_relaxed_fwd(jwf_ctx* ctx, const float* d_pun, const float* d_pburn,
                                const float* d_mask, float* d_pun_out, float* d_pburn_out,
                                void* stream);

/* Adjoint of jwf_step_relaxed_fwd for the same inputs (d_pun, d_pburn,
 * d_mask) and the adjoints d_gun_out, d_gburn_out of its outputs.  Writes
 * the adjoints of the inputs to d_gun, d_gburn (float [cells]); writes
 * d_glam[cell] = dL/dlam(v) (float [cells], may be NULL) for
 * jwf_rates_bwd(); adds dL/dp_continue of this step to *d_gpc (one double,
 * may be NULL; deterministic, summed in a fixed order).  Outputs must not
 * alias inputs. */
JWF_API jwf_status jwf_step_relaxed_bwd(jwf_ctx* ctx, const float* d_pun, const float* d_pburn,
                                const float* d_mask, const float* d_gun_out,
                                const float* d_gburn_out, float* d_gun, float* d_gburn,
                                float* d_glam, double* d_gpc, void* stream);

/* Parameter gradient through the rate table over n_steps relaxed steps.
 * With lam(v) = sum_d pb(v - Delta_d) r[v][d] at every step t,
 *   dL/dtheta += sum_t sum_{v,d} glam_t(v) pb_t(v - Delta_d) dr[v][d]/dtheta
 * for theta = [p_base, alpha_w1, alpha_w2, alpha_s, alpha_gamma, mu_veg[C],
 * mu_den[C]] (JWF_GRAD_SIZE doubles at d_gparams, accumulated, fixed
 * summation order).  d_glam, d_pburn: float [n_steps][cells]; d_mask: float
 * [n_steps][cells] or NULL.  The landcover, elevation and wind inputs are
 * those given to jwf_precompute_probs (Eqs. 1-4 are differentiated exactly;
 * a no-fuel source must carry no burning probability). */
JWF_API jwf_status jwf_rates_bwd(jwf_ctx* ctx, int32_t n_steps, const float* d_glam,
                         const float* d_pburn, const float* d_mask, const uint8_t* d_class,
                         const float* d_dem, const float* d_wind_speed,
                         const float* d_wind_dir, double* d_gparams, void* stream);

/* n_steps relaxed steps in one call (one kernel launch per step, no host
 * work in between).  Forward: d_pun_out / d_pburn_out are [n_steps][cells],
 * row t the state after step t, which starts from row t - 1 (from d_pun /
 * d_pburn for t = 0); d_masks is [n_steps][cells] or NULL.  The outputs must
 * not overlap the inputs.  Same requirements as jwf_step_relaxed_fwd. */
JWF_API jwf_status jwf_relaxed_fwd_steps(jwf_ctx* ctx, int32_t n_steps, const float* d_pun,
                                         const float* d_pburn, const float* d_masks, float* d_pun_out,
                                         float* d_pburn_out, void* stream);

/* Adjoint of n_steps (>= 1) steps in reverse order: d_pun / d_pburn are
 * [n_steps][cells], row t the state before step t; d_gun_out / d_gburn_out
 * the adjoints of the state after step n_steps - 1; d_gun / d_gburn receive
 * the adjoints of the state before step 0; d_glam ([n_steps][cells], row t
 * for step t, or NULL) and d_gpc as in jwf_step_relaxed_bwd.  Uses the
 * context's adjoint scratch (JWF_KEEP_RATES); outputs must not overlap inputs. */
JWF_API jwf_status jwf_relaxed_bwd_steps(jwf_ctx* ctx, int32_t n_steps, const float* d_pun,
                                         const float* d_pburn, const float* d_masks,
                                         const float* d_gun_out, const float* d_gburn_out, float* d_gun,
                                         float* d_gburn, float* d_glam, double* d_gpc, void* stream);

/* The two halves of jwf_rates_bwd, for a backward pass that contracts once:
 * jwf_rates_accumulate adds the rate adjoint of n_steps relaxed steps,
 *   d_gr[v][d] += sum_t glam_t(v) pb_t(v - Delta_d)     (float [cells][8]),
 * summing the chunk in step order before adding (d_glam, d_pburn, d_mask as
 * in jwf_rates_bwd); jwf_rates_contract adds
 *   dL/dtheta += sum_{v,d} d_gr[v][d] dr[v][d]/dtheta
 * to d_gparams (JWF_GRAD_SIZE doubles, fixed summation order).  Calling
 * accumulate on fixed step chunks and contract once gives a result that does
 * not depend on how the steps were recomputed (checkpointing). */
JWF_API jwf_status jwf_rates_accumulate(jwf_ctx* ctx, int32_t n_steps, const float* d_glam,
                                        const float* d_pburn, const float* d_mask, float* d_gr,
                                        void* stream);
JWF_API jwf_status jwf_rates_contract(jwf_ctx* ctx, const float* d_gr, const uint8_t* d_class,
                                      const float* d_dem, const float* d_wind_speed,
                                      const float* d_wind_dir, double* d_gparams, void* stream);

/* ---- no-allocation variant ------------------------------------------------ */

/* Largest batch, in cells (n_envs * H * W), that
 * jwf_step_relaxed_bwd_noalloc accepts. */
#define JWF_NOALLOC_MAX_CELLS (1 << 22)

/* The adjoint step of jwf_step_relaxed_bwd for a uniform batch of n_envs
 * grids of H x W cells, without a context and without allocating device
 * memory.  The paper has no counterpart: this entry point exists for callers
 * that cannot call cudaMalloc -- code running inside another framework's
 * custom operator, which hands over its buffers and forbids allocation while
 * the operator runs, and real-time loops that must not allocate once they
 * have started.
 *
 * Buffers are the caller's, laid out as on the context path: d_r float
 * [cells][8] rate table (e.g. the one jwf_get_probs returns); d_pun, d_pburn,
 * d_gun_out, d_gburn_out float [cells]; d_mask float [cells] or NULL;
 * outputs d_gun, d_gburn float [cells]; *d_gpc (one double, or NULL)
 * accumulates dL/dp_continue.  The results are those of jwf_step_relaxed_bwd
 * on the same inputs.
 *
 * Scratch: one file-scope device array of about 16 MiB (one float per cell
 * for JWF_NOALLOC_MAX_CELLS cells, plus reduction partial sums) that every
 * GPU loading the library holds until the process exits.  Errors: JWF_EINVAL
 * when n_envs * H * W exceeds JWF_NOALLOC_MAX_CELLS, for null pointers,
 * p_continue outside [0, 1], or an output buffer (d_gun, d_gburn, d_gpc)
 * that shares a byte with an input or with another output (sizes as above);
 * JWF_ECUDA when the device or a launch fails.  Every call looks up the
 * array's device address on the current device; the first lookup on a device
 * loads the library's device code there, so make the first call on each
 * device before any stream capture.  All calls share the array, which keeps the
 * last call's contents: calls that overlap on the GPU (on different streams
 * or from different host threads) race, so the caller must serialise them. */
JWF_API jwf_status jwf_step_relaxed_bwd_noalloc(int32_t n_envs, int32_t H, int32_t W,
                                                const float* d_r, float p_continue,
                                                const float* d_pun, const float* d_pburn,
                                                const float* d_mask, const float* d_gun_out,
                                                const float* d_gburn_out, float* d_gun,
                                                float* d_gburn, double* d_gpc, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* JWF_H */
