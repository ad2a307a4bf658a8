/*
 * jwf_oracle.c -- CPU oracle for the stochastic cellular-automaton wildfire
 * model of JaxWildfire (arXiv 2512.06102, Section 3).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The product path (the
 * CUDA library and its Python binding) shares no code with it and never calls
 * it.
 *
 * Plain, slow and single-threaded on purpose: every cell, every direction and
 * every random draw is visited in the order the model defines it, so that a
 * reader can check each line against the paper.
 *
 * Contents
 *   orc_philox4x32_10   Philox4x32-10 counter-based generator, written from
 *                       Salmon, Moraes, Dror & Shaw, "Parallel random numbers:
 *                       as easy as 1, 2, 3" (SC'11), Section 3 / Fig. 2.
 *   orc_uniform24       24-bit uniform in [0,1) from one Philox output word.
 *   orc_drop_mask       3x3 (radius-R) air-tanker drop expanded to a cell mask
 *                       (Section 4: water turns burning cells into burned).
 *   orc_discrete_step   one synchronous step F_t -> F_{t+1} of one grid
 *                       (Section 3, "Stochastic update", Eq. 4 factorised per
 *                       burning neighbour; see below).
 *   orc_discrete_rollout
 *                       k steps of a batch of (possibly ragged) grids with
 *                       per-step drops, per-env counts, done flags and
 *                       optional auto-reset.
 *   orc_discrete_rollout_masks
 *                       the same with each step's action as a cell mask.
 *
 * Cell states (uint8): 0 no fuel (an unburned cell with mu_den = -1, which can
 * never ignite), 1 can burn (unburned, fuel present), 2 burning, 3 burned.
 *
 * Directions d = 0..7 point from a source u to a target v = u + Delta_d.  The
 * angle of Delta_d is d * 45 degrees, east = 0, counting counter-clockwise
 * (Section 3, below Eq. 2).  Grid rows grow southward, so "north" is row - 1:
 *     d : 0=E 1=NE 2=N 3=NW 4=W 5=SW 6=S 7=SE
 *     column step  dx = { 1, 1, 0,-1,-1,-1, 0, 1}
 *     row step     dr = { 0,-1,-1,-1, 0, 1, 1, 1}
 *
 * Probability table q[v][d] (float): the probability that the burning source
 * u = v - Delta_d ignites target v in one step.  By Eq. 4,
 *     P(v ignites) = 1 - exp(-gamma(v) * sum_u b(u) phi(u, Delta_{u->v}))
 *                  = 1 - prod_{burning u} exp(-gamma(v) phi(u, .)),
 * so drawing one independent Bernoulli per burning neighbour with
 * q = 1 - exp(-gamma(v) phi(u, .)) and igniting when any succeeds has exactly
 * the law of Eq. 4.  The table is an input (it is computed in FP64 elsewhere
 * and rounded to float), so this file holds no floating-point model
 * arithmetic beyond the comparison u < q.
 *
 * Random numbers.  Every draw is Philox4x32-10 with
 *     key     = (seed & 0xffffffff, seed >> 32)
 *     counter = (y * W + x, t, env, 4 * episode + slot)
 * where t is the 0-based index of the step being computed (F_t -> F_{t+1}).
 * slot 0 words 0..3 -> spread draws for directions 0..3,
 * slot 1 words 0..3 -> spread draws for directions 4..7,
 * slot 2 word 0     -> the "remain burning" draw of a burning cell,
 * slot 3            -> reserved.
 * A draw succeeds when its uniform u = (word >> 8) * 2^-24 (exact in float) is
 * strictly below the probability (float compare), so probability 0 never fires
 * and probability 1 always fires.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static const int ORC_DX[8] = {1, 1, 0, -1, -1, -1, 0, 1};
static const int ORC_DR[8] = {0, -1, -1, -1, 0, 1, 1, 1};

/* ---------------------------------------------------------------------------
 * Philox4x32-10 (Salmon et al., SC'11).  One round maps counter (c0,c1,c2,c3)
 * and key (k0,k1) to
 *     (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),  hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0))
 * with multipliers M0 = 0xD2511F53, M1 = 0xCD9E8D57; between rounds the key is
 * bumped by the Weyl constants (0x9E3779B9, 0xBB67AE85).  Ten rounds.
 * ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Batch form for tests: n counters [n][4] -> outputs [n][4], one key. */
void orc_philox4x32_10_batch(int64_t n, const uint32_t* ctr, const uint32_t key[2], uint32_t* out)
{
    for (int64_t i = 0; i < n; ++i) orc_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

float orc_uniform24(uint32_t word)
{
    return (float)(word >> 8) * 0x1p-24f;
}

/* One uniform for (cell c0, step t, env, episode, slot, word). */
static float orc_draw(uint64_t seed, uint32_t cell, uint32_t t, uint32_t env,
                      uint32_t episode, uint32_t slot, int word)
{
    uint32_t ctr[4] = {cell, t, env, 4u * episode + slot};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return orc_uniform24(out[word]);
}

/* Drop of radius R centred on (cx, cy) (column, row), clipped to the grid.
 * A centre with cx < 0 or cy < 0 means "no drop this step". */
void orc_drop_mask(int H, int W, int cx, int cy, int R, uint8_t* mask)
{
    memset(mask, 0, (size_t)H * (size_t)W);
    if (cx < 0 || cy < 0) return;
    for (int y = cy - R; y <= cy + R; ++y)
        for (int x = cx - R; x <= cx + R; ++x)
            if (y >= 0 && y < H && x >= 0 && x < W) mask[(size_t)y * W + x] = 1;
}

/* ---------------------------------------------------------------------------
 * One synchronous step of one grid (Section 3 "Stochastic update", plus the
 * tanker action of Section 4 applied first):
 *   1. action: a burning cell under the mask becomes burned;
 *   2. from the post-action grid, every can-burn cell v ignites when at least
 *      one burning neighbour u = v - Delta_d succeeds with probability
 *      q[v][d]; every burning cell stays burning with probability p_continue,
 *      otherwise becomes burned; no-fuel and burned cells do not change.
 * Cells outside the grid are absent (no sparks enter or leave).
 * F_in and F_out must not alias.  Writes the post-step counts of burning and
 * burned cells.
 * ------------------------------------------------------------------------- */
void orc_discrete_step(int H, int W, const uint8_t* F_in, uint8_t* F_out,
                       const float* q, float p_continue, const uint8_t* mask,
                       uint64_t seed, uint32_t env, uint32_t t, uint32_t episode,
                       int32_t* n_burning, int32_t* n_burnt)
{
    size_t n = (size_t)H * (size_t)W;
    uint8_t* Fa = (uint8_t*)malloc(n);
    /* 1. tanker action on F_t */
    for (size_t i = 0; i < n; ++i) {
        uint8_t s = F_in[i];
        if (mask != NULL && mask[i] && s == 2) s = 3;
        Fa[i] = s;
    }
    /* 2. spread and burn-out from the post-action grid */
    int32_t burning = 0, burnt = 0;
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            size_t v = (size_t)y * W + x;
            uint32_t cell = (uint32_t)v;
            uint8_t s = Fa[v], s_next = s;
            if (s == 1) {
                int ignite = 0;
                for (int d = 0; d < 8; ++d) {
                    int ux = x - ORC_DX[d];
                    int uy = y - ORC_DR[d];
                    if (ux < 0 || ux >= W || uy < 0 || uy >= H) continue;
                    if (Fa[(size_t)uy * W + ux] != 2) continue;
                    float u = orc_draw(seed, cell, t, env, episode, (uint32_t)(d / 4), d % 4);
                    if (u < q[v * 8 + d]) ignite = 1;
                }
                s_next = ignite ? 2 : 1;
            } else if (s == 2) {
                float u = orc_draw(seed, cell, t, env, episode, 2u, 0);
                s_next = (u < p_continue) ? 2 : 3;
            }
            F_out[v] = s_next;
            if (s_next == 2) ++burning;
            if (s_next == 3) ++burnt;
        }
    }
    free(Fa);
    if (n_burning) *n_burning = burning;
    if (n_burnt) *n_burnt = burnt;
}

/* ---------------------------------------------------------------------------
 * k steps of a batch of grids.  Env e has shape H[e] x W[e] and its cells start
 * at offset off[e] in F, F0 (cell-major) and at 8 * off[e] in q.
 *   drops   : int32 [k][N][2] (column, row) drop centres, radius R; NULL = none
 *   t, episode : int32 [N], updated in place
 *   t_max   : done when the post-step t reaches t_max (<= 0: no limit)
 *   auto_reset : when an env is done after a step, F_e := F0_e, t := 0,
 *                episode += 1 (the reported counts are the pre-reset ones)
 *   burning, burnt : int32 [k][N] outputs (may be NULL); done : uint8 [k][N]
 *   env_ids : int32 [N] env index used in the random-number counter of each
 *             grid (NULL: its position e), so that a sample of a larger batch
 *             draws the same numbers as in the full batch
 * Done also holds when the post-step grid has no burning cell.
 * ------------------------------------------------------------------------- */
static void rollout(int N, const int32_t* H, const int32_t* W, const int64_t* off,
                    uint8_t* F, const uint8_t* F0, const float* q, float p_continue,
                    const int32_t* drops, const uint8_t* masks, int64_t cells, int R, uint64_t seed,
                    int32_t* t, int32_t* episode, int k, int t_max, int auto_reset,
                    int32_t* burning, int32_t* burnt, uint8_t* done, const int32_t* env_ids)
{
    for (int step = 0; step < k; ++step) {
        for (int e = 0; e < N; ++e) {
            size_t n = (size_t)H[e] * (size_t)W[e];
            uint8_t* Fe = F + off[e];
            uint8_t* tmp = (uint8_t*)malloc(n);
            uint8_t* mask = NULL;
            if (drops != NULL) {
                const int32_t* c = drops + ((size_t)step * N + e) * 2;
                mask = (uint8_t*)malloc(n);
                orc_drop_mask(H[e], W[e], c[0], c[1], R, mask);
            } else if (masks != NULL) {
                mask = (uint8_t*)malloc(n);
                memcpy(mask, masks + (size_t)step * (size_t)cells + (size_t)off[e], n);
            }
            int32_t nb = 0, nd = 0;
            uint32_t env = env_ids != NULL ? (uint32_t)env_ids[e] : (uint32_t)e;
            orc_discrete_step(H[e], W[e], Fe, tmp, q + 8 * off[e], p_continue, mask, seed,
                              env, (uint32_t)t[e], (uint32_t)episode[e], &nb, &nd);
            memcpy(Fe, tmp, n);
            free(tmp);
            free(mask);
            t[e] += 1;
            int is_done = (nb == 0) || (t_max > 0 && t[e] >= t_max);
            if (burning) burning[(size_t)step * N + e] = nb;
            if (burnt) burnt[(size_t)step * N + e] = nd;
            if (done) done[(size_t)step * N + e] = (uint8_t)is_done;
            if (is_done && auto_reset) {
                memcpy(Fe, F0 + off[e], n);
                t[e] = 0;
                episode[e] += 1;
            }
        }
    }
}

void orc_discrete_rollout(int N, const int32_t* H, const int32_t* W, const int64_t* off,
                          uint8_t* F, const uint8_t* F0, const float* q, float p_continue,
                          const int32_t* drops, int R, uint64_t seed,
                          int32_t* t, int32_t* episode, int k, int t_max, int auto_reset,
                          int32_t* burning, int32_t* burnt, uint8_t* done, const int32_t* env_ids)
{
    rollout(N, H, W, off, F, F0, q, p_continue, drops, NULL, 0, R, seed, t, episode, k, t_max, auto_reset,
            burning, burnt, done, env_ids);
}

/* The same rollout with the tanker action of each step given as a cell mask:
 * masks uint8 [k][cells] (cells = the batch's total), nonzero = water on the
 * cell at that step (a burning cell there becomes burned before the spread). */
void orc_discrete_rollout_masks(int N, const int32_t* H, const int32_t* W, const int64_t* off,
                                uint8_t* F, const uint8_t* F0, const float* q, float p_continue,
                                const uint8_t* masks, int64_t cells, uint64_t seed,
                                int32_t* t, int32_t* episode, int k, int t_max, int auto_reset,
                                int32_t* burning, int32_t* burnt, uint8_t* done, const int32_t* env_ids)
{
    rollout(N, H, W, off, F, F0, q, p_continue, NULL, masks, cells, 1, seed, t, episode, k, t_max, auto_reset,
            burning, burnt, done, env_ids);
}

/* ---------------------------------------------------------------------------
 * Monte-Carlo helper for the statistical pins: n_trials independent copies of
 * one step of the same grid; trial i uses env index i, so each trial reads its
 * own Philox stream.  out: uint8 [n_trials][H*W] post-step states.
 * ------------------------------------------------------------------------- */
void orc_mc_outcomes(int H, int W, const uint8_t* F, const float* q, float p_continue,
                     const uint8_t* mask, uint64_t seed, uint32_t t, uint32_t episode,
                     int64_t n_trials, uint8_t* out)
{
    size_t n = (size_t)H * (size_t)W;
    for (int64_t i = 0; i < n_trials; ++i)
        orc_discrete_step(H, W, F, out + (size_t)i * n, q, p_continue, mask, seed,
                          (uint32_t)i, t, episode, NULL, NULL);
}
