// jwf_internal.cuh -- shared definitions of libjwf's translation units.
//
// Device-side building blocks (directions, Philox4x32-10, 24-bit uniforms),
// the context struct and the host-side launchers that jwf_api.cu calls.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/jwf.h"

#define JWF_MAX_CLASSES 64

// ---------------------------------------------------------------------------
// Directions: Delta_d has angle d*45 degrees, east = 0, counter-clockwise
// (Section 3, below Eq. 2).  Rows grow southward.  The source of target
// (row y, column x) in direction d is (y - DR[d], x - DX[d]).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int jwf_dx(int d) {
    return (d == 0 || d == 1 || d == 7) ? 1 : (d == 3 || d == 4 || d == 5) ? -1 : 0;
}
__host__ __device__ constexpr int jwf_dr(int d) {
    return (d == 1 || d == 2 || d == 3) ? -1 : (d == 5 || d == 6 || d == 7) ? 1 : 0;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
//   (c0,c1,c2,c3) <- (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0))
// with the key bumped by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 jwf_philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c.y ^ k0;
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c.w ^ k1;
        c = make_uint4(n0, (uint32_t)p1, n2, (uint32_t)p0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Tanker action masks travel bit-packed: a row of jwf_mask_row_words(cells)
// 32-bit words per step, cell g of the context at bit g % 32 of word g / 32.
inline __host__ __device__ int64_t jwf_mask_row_words(int64_t cells) { return (cells + 31) / 32; }

// bits of a mask row for cells [g, g + n) of the context (0 < n <= 32), cell
// g + i at bit i; reads only words that hold those cells
__device__ __forceinline__ uint32_t mask_run(const uint32_t* __restrict__ row, int64_t g, int n) {
    const int64_t w = g >> 5;
    const int sh = (int)(g & 31);
    uint32_t v = __ldg(row + w) >> sh;
    if (sh + n > 32) v |= __ldg(row + w + 1) << (32 - sh);
    return n >= 32 ? v : v & ((1u << n) - 1u);
}

// Uniform in [0,1) with 24 random bits; exact in float.
__device__ __forceinline__ float jwf_u24(uint32_t w) { return (float)(w >> 8) * 0x1p-24f; }

// cp.async (asynchronous global -> shared copies, completed by groups): the
// tiled kernels stage the next tile or step while computing the current one.
__device__ __forceinline__ void jwf_cp_async4(float* dst, const float* src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void jwf_cp_async16(float* dst, const float* src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void jwf_cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void jwf_cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void jwf_cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// ---------------------------------------------------------------------------
// TMA (cp.async.bulk.tensor) with an mbarrier: the tiled step stages its
// region (tile plus halo) with one 2-D tensor copy.  A tensor map is the
// 128-byte object cuTensorMapEncodeTiled writes; the kernels only pass its
// global address to the copy instruction.
// ---------------------------------------------------------------------------
struct alignas(64) JwfTmap {
    unsigned long long w[16];
};

__device__ __forceinline__ uint32_t jwf_smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void jwf_mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(jwf_smem_u32(bar)), "r"(count) : "memory");
    // make the initialised barrier visible to the asynchronous (TMA) proxy
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void jwf_mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(jwf_smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool jwf_mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(jwf_smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0u;
}
__device__ __forceinline__ uint64_t jwf_globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}
// Wait for phase `parity` of the barrier for at most `ns` nanoseconds;
// false when the wait gave up.
__device__ __forceinline__ bool jwf_mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t ns) {
    const uint64_t t0 = jwf_globaltimer();
    while (!jwf_mbar_try_wait(bar, parity))
        if (jwf_globaltimer() - t0 > ns) return false;
    return true;
}
// order this thread's earlier shared-memory accesses before later TMA accesses
__device__ __forceinline__ void jwf_fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
// 2-D tile load global -> shared, completion counted on the barrier (bytes);
// x (innermost, elements) must be a multiple of 16 bytes, y is any row
__device__ __forceinline__ void jwf_tma_load_2d(void* dst, const JwfTmap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
            jwf_smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(jwf_smem_u32(bar))
        : "memory");
}
// 2-D tile store shared -> global (elements outside the tensor are not written);
// x >= 0 and a multiple of 16 bytes, y >= 0
__device__ __forceinline__ void jwf_tma_store_2d(const JwfTmap* map, int x, int y, const void* src) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];\n" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(jwf_smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void jwf_bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void jwf_bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }

// ---------------------------------------------------------------------------
// Parameters as the kernels see them (by value).
// ---------------------------------------------------------------------------
struct JwfDevParams {
    float p_base, alpha_w1, alpha_w2, alpha_s, alpha_gamma, p_continue, cell_size;
    int32_t n_classes;
    float mu_veg[JWF_MAX_CLASSES];
    float mu_den[JWF_MAX_CLASSES];
};

// Per-cell kernels walk blocks of JWF_TILE consecutive cells of one env.
#define JWF_TILE 256
// The plain step: a thread steps row segments of JWF_PLAIN_SEG cells, a block
// JWF_PLAIN_SEGS_PER_THREAD x JWF_TILE consecutive segments of one env.
#define JWF_PLAIN_SEG 16
#define JWF_PLAIN_SEGS_PER_THREAD 4
// The tiled relaxed kernels walk 2-D tiles of JWF_RT_ROWS x JWF_RT_COLS cells.
#define JWF_RT_ROWS 16
#define JWF_RT_COLS 64
// The two-step relaxed forward walks tiles of JWF_R2_ROWS x JWF_R2_COLS cells.
#define JWF_R2_ROWS 16
#define JWF_R2_COLS 32
// The relaxed adjoint sweeps strips of JWF_SW_COLS output columns (one warp,
// a halo column on each side) down JWF_SW_ROWS rows.
#define JWF_SW_COLS 30
#define JWF_SW_ROWS 32
// The two-step adjoint sweeps strips of JWF_SW2_COLS output columns (two halo
// columns on each side) down JWF_SW2_ROWS rows.
#define JWF_SW2_COLS 28
#define JWF_SW2_ROWS 32

// A size class of envs run by one resident launch: envs order[start ..
// start + count), the largest shape in it, and its block size (0: by size).
struct JwfGroup {
    int32_t start = 0, count = 0, maxH = 0, maxW = 0, threads = 0, size_class = 0;
};
#define JWF_MAX_GROUPS 4

struct jwf_ctx {
    int device = 0;
    int num_sms = 0;
    int32_t N = 0;
    int64_t cells = 0;
    int32_t maxH = 0, maxW = 0;
    int64_t max_env_cells = 0;
    int32_t n_classes = 0;
    uint64_t seed = 0;
    int32_t t_max = 0;
    int32_t drop_radius = 1;
    uint32_t flags = 0;
    std::vector<int32_t> H, W;
    std::vector<int64_t> off;            // N + 1

    // device memory owned by the context
    int32_t* d_H = nullptr;
    int32_t* d_W = nullptr;
    int64_t* d_off = nullptr;
    int32_t* d_order = nullptr;          // env processing order, largest first
    int32_t* d_order_dyn = nullptr;      // [N] order of the second part of a split resident launch
    int32_t* d_lastb = nullptr;          // [N] burning cells after the first part
    int32_t reorder_steps = 12;          // split resident launches after this many steps (0: never)
    int2* d_tiles = nullptr;             // (env, first local cell) per JWF_TILE block
    int64_t n_tiles = 0;
    int2* d_ptiles = nullptr;            // (env, first row segment) per plain-step block
    int64_t n_ptiles = 0;
    uint8_t* d_state[2] = {nullptr, nullptr};
    int cur = 0;                         // index of the current state buffer
    uint8_t* d_F0 = nullptr;
    float* d_q = nullptr;
    float* d_r = nullptr;
    int32_t* d_t = nullptr;
    int32_t* d_episode = nullptr;
    int32_t* d_cnt = nullptr;            // [2][N] per-step counts (plain path)
    uint8_t* d_flag = nullptr;           // [N] per-env done/reset flags
    uint32_t* d_status = nullptr;        // device error word
    uint32_t* d_queue = nullptr;         // [2] work queue cursor, exit counter
    double* d_partials = nullptr;        // deterministic reduction scratch
    int64_t partial_cap = 0;             // doubles available in d_partials
    uint32_t* d_red_counter = nullptr;   // blocks finished (last-block reduction)
    float* d_glam = nullptr;             // [cells] adjoint scratch of the relaxed step
    float* d_adj = nullptr;              // [2][cells] adjoint ping-pong of the multi-step relaxed adjoint
    float* d_gr = nullptr;               // [cells][8] rate-adjoint scratch of jwf_rates_bwd
    unsigned long long* d_pairs = nullptr;  // caller's instrumentation counter (not owned)
    float2* d_wexp = nullptr;            // [N][8] wind exponent (hi, lo) scratch of the table build
    // terrain borrowed from the caller for the fused step (jwf_set_terrain)
    const uint8_t* t_cls = nullptr;
    const float* t_dem = nullptr;
    const float* t_ws = nullptr;
    const float* t_wd = nullptr;
    bool have_terrain = false;
    // tiled path: (env, tile row, tile column) per tile, per-env tile layout,
    // per-tile activity (ping-pong), buffers-in-sync flags, burned counts,
    // and the per-round count scratch [16][2][N]
    int4* d_tiles4 = nullptr;
    int4* d_env_tiles = nullptr;
    int64_t n_tiles4 = 0;
    int4* d_rtiles = nullptr;            // (env, first row, first column) per relaxed 2-D tile
    int64_t n_rtiles = 0;
    int4* d_r2tiles = nullptr;           // (env, first row, first column) per two-step forward tile
    int64_t n_r2tiles = 0;
    int4* d_stiles = nullptr;            // (env, first row, first column) per adjoint sweep strip
    int64_t n_stiles = 0;
    int4* d_s2tiles = nullptr;           // ... per two-step adjoint sweep strip
    int64_t n_s2tiles = 0;
    int relaxed_kernel = 0;              // 0: tiled (fused adjoint), 1: plain (two-pass adjoint)
    uint16_t* d_tact[2] = {nullptr, nullptr};
    int tact_cur = 0;
    int tplan_cur = 0;                   // which of the two round plans (and count scratch) the next round uses
    uint8_t* d_tsync = nullptr;
    // tensor maps of the tiled step, per env: [2 buffers][region box, tile box][N]
    // (built at creation for envs whose rows start 16-byte aligned), and the
    // per-env flag that they exist
    JwfTmap* d_tmaps = nullptr;
    uint8_t* d_tma_ok = nullptr;
    bool tma = false;
    bool use_tma = true;                 // jwf_set_tile_copy: TMA (default) or plain loads
    uint64_t tma_wait_ns = 2000000000ull;   // a tensor copy that takes 2 s has failed
    bool tma_diag_no_copy = false;       // diagnostics (jwf_set_tile_copy_wait): the waits run out
    int32_t* d_tburnt = nullptr;
    int32_t* d_tcnt = nullptr;
    // per-round plan of the persistent tiled step: [0] active tiles, [1]
    // quiet tiles to copy once, [2] work cursor, [3] unused, then the burned
    // cells of each env's quiet tiles [N], the active list and the copy list
    // [n_tiles4 each]; the header and the per-env sums are zero between rounds
    int32_t* d_tplan = nullptr;
    int tiled_grid[2] = {0, 0};          // persistent CTAs of the tiled step (table, fused)
    bool tiles_valid = false;
    int32_t round_steps = 16;            // steps per tiled launch (1..16)
    // size classes of the resident path and the streams/events they fork onto
    std::vector<JwfGroup> groups;
    cudaStream_t side[JWF_MAX_GROUPS] = {};
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_join[JWF_MAX_GROUPS] = {};
    bool wexp_stale = true;              // parameters changed since d_wexp was built
    // wind time series (fused kernels): [wser_n][N][8] wind exponents of the
    // series' steps, from borrowed [wser_n][N] speed and direction arrays
    float2* d_wser = nullptr;
    int64_t wser_cap = 0;                // float2 entries allocated
    int32_t wser_n = 0;                  // steps in the series (0: static wind)
    const float* s_ws = nullptr;
    const float* s_wd = nullptr;
    bool wser_stale = false;
    uint8_t* hist = nullptr;             // during a recording jwf_step: [k][cells] states after each step
    bool hist_packed = false;            // hist rows are 2-bit packed, jwf_packed_bytes(cells) apart
    bool packed_aligned = false;         // every env starts on a 32-cell boundary and has W % 32 == 0
    int32_t* d_agent_drops = nullptr;    // [N][2] drop centres of an agent step
    int32_t* d_agent_cnt = nullptr;      // [N] burning cells after an agent step
    uint8_t* d_agent_done = nullptr;     // [N] done flags of an agent step

    JwfDevParams P{};
    bool have_params = false, have_table = false, have_rates = false, have_state = false;
    jwf_kernel kernel = JWF_KERNEL_AUTO;
    int threads_per_env = 0;             // 0: chosen by size
    std::string last_error;
};

// Device status word bits.
#define JWF_DEVERR_TMA 0x2u        // a tensor-copy wait gave up (the tile was not stepped)

// ---------------------------------------------------------------------------
// Launchers (host functions; each returns cudaGetLastError() of its launch).
// ---------------------------------------------------------------------------
cudaError_t jwf_launch_wind_exponent(const jwf_ctx* c, const float* ws, const float* wd, cudaStream_t s);
cudaError_t jwf_launch_wind_series(jwf_ctx* c, cudaStream_t s);
cudaError_t jwf_launch_agent_act(const jwf_ctx* c, const int32_t* actions, int32_t* agent, cudaStream_t s);
cudaError_t jwf_launch_agent_post(const jwf_ctx* c, int mode, int32_t* agent, int32_t water0, int random_fire,
                                  float burn_penalty, float* reward, int32_t obs_k, uint8_t* obs, cudaStream_t s);
cudaError_t jwf_launch_agent_warp(const jwf_ctx* c, bool fused, const int32_t* actions, int32_t* agent,
                                  int32_t water0, int random_fire, float burn_penalty, float* reward, uint8_t* done,
                                  int32_t obs_k, uint8_t* obs, cudaStream_t s);
cudaError_t jwf_launch_state_planes(int64_t n, const uint8_t* states, float* pun, float* pburn, cudaStream_t s);
cudaError_t jwf_launch_prob_check(const jwf_ctx* c, int64_t n, const uint8_t* cv, const uint8_t* cu,
                                  const float* zv, const float* zu, const float* wexp, const int32_t* dir,
                                  float* out, cudaStream_t s);
cudaError_t jwf_launch_prob_table(const jwf_ctx* c, const uint8_t* cls, const float* dem,
                                  const float* ws, const float* wd, cudaStream_t s);
cudaError_t jwf_launch_rates_accumulate(const jwf_ctx* c, int32_t n_steps, const float* glam,
                                        const float* pburn, const float* mask, float* gr, cudaStream_t s);
cudaError_t jwf_launch_rates_contract(jwf_ctx* c, const float* gr, const uint8_t* cls, const float* dem,
                                      const float* ws, const float* wd, double* gparams, cudaStream_t s);
cudaError_t jwf_launch_rates_bwd(jwf_ctx* c, int32_t n_steps, const float* glam,
                                 const float* pburn, const float* mask, const uint8_t* cls,
                                 const float* dem, const float* ws, const float* wd,
                                 double* gparams, cudaStream_t s);

cudaError_t jwf_launch_load(jwf_ctx* c, const uint8_t* F0, cudaStream_t s);
// 2-bit packed states: cell i sits in bits 2(i mod 4), 2(i mod 4) + 1 of byte
// i / 4.  A packed row of `cells` states takes jwf_packed_bytes(cells) bytes
// (rounded up to 16 so that consecutive rows stay 16-byte aligned).
inline int64_t jwf_packed_bytes(int64_t cells) { return ((cells + 3) / 4 + 15) / 16 * 16; }
cudaError_t jwf_launch_pack(int64_t n, const uint8_t* states, uint8_t* packed, cudaStream_t s);
cudaError_t jwf_launch_unpack(int64_t n, const uint8_t* packed, uint8_t* states, cudaStream_t s);
cudaError_t jwf_launch_load_packed(jwf_ctx* c, const uint8_t* P0, cudaStream_t s);
// record the current state as history row `row` (u8 copy or packed)
cudaError_t jwf_record_row(jwf_ctx* c, int64_t row, cudaStream_t s);
cudaError_t jwf_launch_reset(jwf_ctx* c, const uint8_t* env_mask, cudaStream_t s);
cudaError_t jwf_launch_action(jwf_ctx* c, const uint8_t* mask, cudaStream_t s);
// the step launchers take the steps' actions as drop centres [k][N][2] or as
// mask bit rows [k][jwf_mask_row_words(cells)] (at most one of the two)
cudaError_t jwf_launch_step_plain(jwf_ctx* c, int32_t k, const int32_t* drops, const uint32_t* masks,
                                  int32_t* burning, int32_t* burnt, uint8_t* done, cudaStream_t s);
cudaError_t jwf_launch_step_resident(jwf_ctx* c, int32_t k, const int32_t* drops, const uint32_t* masks,
                                     int32_t* burning, int32_t* burnt, uint8_t* done,
                                     cudaStream_t s);
cudaError_t jwf_launch_step_tiled(jwf_ctx* c, int32_t k, const int32_t* drops, const uint32_t* masks,
                                  int32_t* burning, int32_t* burnt, uint8_t* done, bool fused, cudaStream_t s);
cudaError_t jwf_launch_pack_masks(int32_t n_rows, int64_t cells, const uint8_t* masks, uint32_t* bits,
                                  cudaStream_t s);
// tensor maps of the tiled step's TMA copies (c->d_tmaps, c->d_tma_ok,
// c->tma); envs that do not qualify, or a driver without the encoder, keep
// the plain loads
cudaError_t jwf_build_tile_maps(jwf_ctx* c);
int jwf_tile_rows();
int jwf_tile_cols();
// shared memory a resident launch needs for env shape (H, W) with `threads`
size_t jwf_resident_smem(int32_t H, int32_t W, int threads);
int jwf_resident_threads(int32_t H, int32_t W);

// two relaxed steps in one pass (tiled kernels only): the state after step t
// (pun1, pburn1) and after step t + 1 (pun2, pburn2); masks of the two steps
// or null
cudaError_t jwf_launch_relaxed_fwd2(const jwf_ctx* c, const float* pun, const float* pburn, const float* mask0,
                                    const float* mask1, float* pun1, float* pburn1, float* pun2, float* pburn2,
                                    cudaStream_t s);
cudaError_t jwf_launch_relaxed_fwd(const jwf_ctx* c, const float* pun, const float* pburn,
                                   const float* mask, float* pun_out, float* pburn_out,
                                   cudaStream_t s);
// two adjoint steps in one pass (tiled kernels only): states before step t
// (pun0, pburn0) and before step t + 1 (pun1, pburn1), masks of the two steps
// or null, the adjoints of the state after step t + 1 in, of the state before
// step t out, and dL/dlam of both steps
cudaError_t jwf_launch_relaxed_bwd2(jwf_ctx* c, const float* pun0, const float* pburn0, const float* mask0,
                                    const float* pun1, const float* pburn1, const float* mask1,
                                    const float* gun_out, const float* gburn_out, float* gun, float* gburn,
                                    float* glam0, float* glam1, double* gpc, cudaStream_t s);
cudaError_t jwf_launch_relaxed_bwd(jwf_ctx* c, const float* pun, const float* pburn,
                                   const float* mask, const float* gun_out,
                                   const float* gburn_out, float* gun, float* gburn,
                                   float* glam, double* gpc, cudaStream_t s);
