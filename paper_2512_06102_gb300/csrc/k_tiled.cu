// k_tiled.cu -- the tiled, temporally blocked discrete step (Section 3
// "Stochastic update", tanker action of Section 4) for grids larger than
// shared memory: one CTA per tile and round of up to 16 steps, the region
// (tile plus halo) staged by one TMA tensor copy, then stepped as bit planes
// with the same three phases as the resident step.
#include <cuda.h>

#include <type_traits>
#include <vector>

#include "bitplane.cuh"

namespace {

// ---------------------------------------------------------------------------
// Tiled, temporally blocked step for grids that do not fit shared memory.
//
// One CTA per tile of up to kTileRows x kTileCols interior cells and one
// launch per round of kb <= kMaxRound steps.  The CTA loads the tile with a
// halo of kb rows and one 32-cell word of columns on each side (cells outside
// the grid read as no fuel), runs kb steps over the whole region (halo cells
// are recomputed redundantly; after s steps the outer s cells of the region
// are stale, never the interior), then writes the interior to the other state
// buffer.  A tile that holds no burning cell, and none of whose eight
// neighbours holds one within kMaxRound cells of the side or corner they
// share, cannot change this round: it copies its interior to the other buffer
// once and otherwise only reports its counts.
// ---------------------------------------------------------------------------
constexpr int kTileRows = 64, kTileCols = 128, kMaxRound = 16;
constexpr int kRegionRows = kTileRows + 2 * kMaxRound;
constexpr int kRegionWords = kTileCols / 32 + 2;
// chunk flag bytes of one burning buffer (a chunk is 32 words), rounded to words
constexpr int kRegionWordsAll = kRegionRows * kRegionWords;
constexpr int kRegionChunks = (kRegionWordsAll + 31) / 32;
constexpr int kTileFlagBytes = (kRegionChunks + 3) / 4 * 4;
// block-wide queue of the step's work items (burning-cell draws and compared
// pairs); a chunk whose items do not fit is evaluated by its own warp
constexpr int kQCap = 4096;
constexpr uint32_t kTileVoid = 0xffffffffu;   // a voided queue slot (real items have bits 8..13 clear)

struct TileArgs {
    const int32_t* H;
    const int32_t* W;
    const int64_t* off;
    const int4* tiles;           // (env, tile row, tile column, 0)
    const int4* env_tiles;       // per env: (first tile, tiles per row, tile rows, 0)
    int32_t N;
    const uint8_t* Fin;
    uint8_t* Fout;
    const float* q;
    const uint8_t* cls;
    const float* dem;
    const float2* wexp;
    int32_t wser_n;
    const int32_t* drops;        // [kb][N][2] of this round, or null
    const uint32_t* mask;        // [kb][mask_words] action mask bit rows of this round, or null
    int64_t mask_words;
    const int32_t* t;            // step counters at the start of the round
    const int32_t* episode;
    int32_t* cnt;                // [kb][2][N] per-step counts (zeroed before the round)
    const uint16_t* act_in;      // [tiles] where the last round left burning cells (kAct* bits)
    uint16_t* act_out;
    uint8_t* synced;             // [tiles] both buffers hold this tile's interior
    int32_t* tile_burnt;         // [tiles] burned interior cells after the last round
    unsigned long long* counts;
    // TMA: per env, the region-box map of the input buffer and the tile-box
    // maps of both buffers; tma_ok[e] != 0 where they exist (else null)
    const JwfTmap* tm_region;
    const JwfTmap* tm_in_tile;
    const JwfTmap* tm_out_tile;
    const uint8_t* tma_ok;
    uint32_t* status;
    uint64_t wait_ns;            // bound of a tensor-copy wait
    int32_t diag_no_copy;        // diagnostics: arm the barrier but issue no copy (the wait runs out)
    int32_t* plan;               // the round's plan (k_tile_plan): counts, cursor, lists
    int64_t n_tiles;
    int32_t kb;
    int32_t R;
    uint32_t key0, key1;
    float p_continue;
};

// TMA boxes: the region (tile plus kMaxRound rows and one 32-cell word of
// columns on each side) and the tile itself, one byte a cell
constexpr int kBoxCols = kTileCols + 64, kBoxRows = kRegionRows;

// the staged region fits where it is put (ignition, burn-out and queue arrays,
// from a 128-byte boundary)
static_assert((2 * kRegionWordsAll + kQCap) * 4 >= kBoxRows * kBoxCols + 128, "region staging does not fit");

size_t tiled_smem_bytes(int threads) {
    // planes, warp scratch, chunk flags, ignition and burn-out planes, queue,
    // per-warp lists of dealt chunks
    return (size_t)(2 * (kRegionRows + 2) * kRegionWords + 2 * kRegionWordsAll + (threads / 32) * kWarpScratch +
                    2 * kTileFlagBytes / 4 + 2 * kRegionWordsAll + kQCap + (threads / 32) * kRegionChunks) *
           sizeof(uint32_t);
}

// Region-relative drops: the centre (cx, cy) may lie outside the region (even
// at negative coordinates) while its footprint reaches in; `has` is false for
// a step without a drop.
__device__ __forceinline__ uint32_t drop_bits_rel(int y, int w, int cx, int cy, int R, bool has) {
    if (!has || abs(y - cy) > R) return 0u;
    const int lo = max(cx - R - (w << 5), 0), hi = min(cx + R - (w << 5), 31);
    if (lo > hi) return 0u;
    const uint32_t span = (hi - lo == 31) ? 0xffffffffu : ((1u << (hi - lo + 1)) - 1u);
    return span << lo;
}

__device__ void res_action_rel(int RH, int WW, uint32_t* Bp, uint32_t* D, int cx, int cy, int R, bool has) {
    if (!has) return;
    const int y0 = max(cy - R, 0), y1 = min(cy + R, RH - 1);
    const int x0 = max(cx - R, 0), x1 = min(cx + R, (WW << 5) - 1);
    if (y0 > y1 || x0 > x1) return;
    const int w0 = x0 >> 5, w1 = x1 >> 5;
    const int nw = w1 - w0 + 1;
    const int total = (y1 - y0 + 1) * nw;
    for (int j = threadIdx.x; j < total; j += blockDim.x) {
        const int y = y0 + j / nw, w = w0 + j % nw;
        const uint32_t m = drop_bits_rel(y, w, cx, cy, R, true);
        uint32_t* bp = &Bp[(y + 1) * WW + w];
        const uint32_t doused = *bp & m;
        *bp &= ~m;
        D[y * WW + w] |= doused;
    }
}

// Action mask bits of region word (row gy, columns gx0 .. gx0 + 31 of the
// grid), columns and rows outside the grid 0.
__device__ __forceinline__ uint32_t region_mask(const uint32_t* __restrict__ mrow, int64_t off, int gy, int gx0,
                                                int H, int W) {
    if (gy < 0 || gy >= H) return 0u;
    const int c0 = max(gx0, 0), c1 = min(gx0 + 31, W - 1);
    if (c0 > c1) return 0u;
    return mask_run(mrow, off + (int64_t)gy * W + c0, c1 - c0 + 1) << (c0 - gx0);
}

// Tile activity after a round: kActAny = a burning interior cell; the other
// bits = a burning interior cell within kMaxRound cells of an edge (N, S, W,
// E) or of both edges at a corner.  Fire moves at most one cell a step, so in
// a round of kb <= kMaxRound steps a tile's interior can change only if it
// holds a burning cell or a neighbour holds one within kMaxRound cells of
// the side or corner they share.
constexpr uint16_t kActN = 1, kActS = 2, kActW = 4, kActE = 8, kActNW = 16, kActNE = 32, kActSW = 64,
                   kActSE = 128, kActAny = 256;

// bits of region word w inside the column range [c0, c1) of the region
__device__ __forceinline__ uint32_t col_bits(int w, int c0, int c1) {
    const int lo = max(c0 - (w << 5), 0), hi = min(c1 - (w << 5), 32) - 1;
    if (lo > hi) return 0u;
    const uint32_t span = (hi - lo == 31) ? 0xffffffffu : ((1u << (hi - lo + 1)) - 1u);
    return span << lo;
}

// The plan of a round, one thread per tile.  A tile runs the round when it
// holds fire or a neighbour holds fire within kMaxRound cells of the side or
// corner they share (fire moves at most one cell a step): it goes to the
// active list.  Every other tile keeps its interior: its burned cells go to
// its env's sum, its activity for the next round is none, and when the other
// buffer does not hold its interior yet it goes to the copy list.  The plan
// kernel also zeroes the round's per-step count scratch.
struct PlanArgs {
    int64_t n_tiles;
    const int4* tiles;
    const int4* env_tiles;
    const uint16_t* act_in;
    uint16_t* act_out;
    const uint8_t* synced;
    const int32_t* tile_burnt;
    int32_t N;
    int32_t* plan;
    int32_t* cnt;
    int64_t n_cnt;
};

// The plan's work for tile tix (every thread of the grid, full warps).
__device__ __forceinline__ void tile_plan_part(const PlanArgs& p, int64_t tix) {
    const int64_t n_tiles = p.n_tiles;
    const int4* __restrict__ tiles = p.tiles;
    const int4* __restrict__ env_tiles = p.env_tiles;
    const uint16_t* __restrict__ act_in = p.act_in;
    uint16_t* __restrict__ act_out = p.act_out;
    const uint8_t* __restrict__ synced = p.synced;
    const int32_t* __restrict__ tile_burnt = p.tile_burnt;
    const int32_t N = p.N;
    int32_t* __restrict__ plan = p.plan;
    int32_t* __restrict__ cnt = p.cnt;
    const int64_t n_cnt = p.n_cnt;
    for (int64_t i = tix; i < n_cnt; i += (int64_t)gridDim.x * blockDim.x) cnt[i] = 0;
    const int lane = threadIdx.x & 31;
    bool active = false, copy = false;
    if (tix < n_tiles) {
        const int4 tl = tiles[tix];
        const int e = tl.x, tr = tl.y, tc = tl.z;
        const int4 et = env_tiles[e];
        // the bit of neighbour (dy, dx) that faces this tile
        constexpr uint16_t facing[3][3] = {{kActSE, kActS, kActSW}, {kActE, kActAny, kActW}, {kActNE, kActN, kActNW}};
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int r = tr + dy, c = tc + dx;
                if (r >= 0 && r < et.z && c >= 0 && c < et.y)
                    active |= (act_in[et.x + r * et.y + c] & facing[dy + 1][dx + 1]) != 0;
            }
        if (!active) {
            act_out[tix] = 0;
            copy = synced[tix] == 0;
            const int32_t b = tile_burnt[tix];
            if (b != 0) atomicAdd(&plan[4 + e], b);
        }
    }
    const uint32_t am = __ballot_sync(0xffffffffu, active);
    const uint32_t cm = __ballot_sync(0xffffffffu, copy);
    int base_a = 0, base_c = 0;
    if (lane == 0) {
        if (am) base_a = atomicAdd(&plan[0], __popc(am));
        if (cm) base_c = atomicAdd(&plan[1], __popc(cm));
    }
    base_a = __shfl_sync(0xffffffffu, base_a, 0);
    base_c = __shfl_sync(0xffffffffu, base_c, 0);
    const uint32_t below = (1u << lane) - 1u;
    int32_t* act_list = plan + 4 + N;
    if (active) act_list[base_a + __popc(am & below)] = (int32_t)tix;
    if (copy) act_list[n_tiles + base_c + __popc(cm & below)] = (int32_t)tix;
}

__global__ void __launch_bounds__(256) k_tile_plan(const PlanArgs p) {
    tile_plan_part(p, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

// Tile activity and burned interior cells from a state buffer, one CTA per
// tile (after the state changed outside the tiled path): the same activity
// bits a round leaves behind, so that only tiles with fire within reach run
// the next round, and the burned count a quiet tile reports.  The interior is
// copied to the other buffer on the way, so both buffers hold it.
__global__ void __launch_bounds__(256)
k_tile_act_init(const int4* __restrict__ tiles, const int32_t* __restrict__ Hs, const int32_t* __restrict__ Ws,
                const int64_t* __restrict__ offs, const uint8_t* __restrict__ F, uint8_t* __restrict__ Fo,
                uint16_t* __restrict__ act, uint8_t* __restrict__ synced, int32_t* __restrict__ tile_burnt) {
    __shared__ uint32_t s_act;
    __shared__ int32_t s_burnt;
    const int tix = blockIdx.x;
    const int4 tl = tiles[tix];
    const int e = tl.x;
    const int H = Hs[e], W = Ws[e];
    const int ty0 = tl.y * kTileRows, tx0 = tl.z * kTileCols;
    const int TY = min(kTileRows, H - ty0), TX = min(kTileCols, W - tx0);
    const uint8_t* Fe = F + offs[e];
    uint8_t* Foe = Fo + offs[e];
    if (threadIdx.x == 0) {
        s_act = 0u;
        s_burnt = 0;
    }
    __syncthreads();
    constexpr int band = kMaxRound;
    uint32_t a = 0u;
    int nd = 0;
    // one cell's contribution: burned count, activity bits of a burning cell
    auto cell = [&](uint8_t st, int y, int x) {
        nd += st == 3;
        if (st != 2) return;
        const bool n = y < band, so = TY - 1 - y < band, wb = x < band, eb = TX - 1 - x < band;
        a |= kActAny | (n ? kActN : 0) | (so ? kActS : 0) | (wb ? kActW : 0) | (eb ? kActE : 0) |
             (n && wb ? kActNW : 0) | (n && eb ? kActNE : 0) | (so && wb ? kActSW : 0) | (so && eb ? kActSE : 0);
    };
    if (((offs[e] | (int64_t)W) & 15) == 0 && (TX & 15) == 0) {
        // 16 cells a thread: rows start on 16-byte boundaries (tx0 is a multiple of 128)
        const int segs = TX >> 4;
        for (int i = threadIdx.x; i < TY * segs; i += blockDim.x) {
            const int y = i / segs, x0 = (i - y * segs) << 4;
            const int64_t g = (int64_t)(ty0 + y) * W + tx0 + x0;
            const uint4 v = *reinterpret_cast<const uint4*>(Fe + g);
            *reinterpret_cast<uint4*>(Foe + g) = v;
            const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                nd += __popc(__vcmpeq4(w4[k], 0x03030303u)) >> 3;
                const uint32_t b = __vcmpeq4(w4[k], 0x02020202u);
                if (b == 0u) continue;
                for (int j = 0; j < 4; ++j)
                    if ((b >> (8 * j)) & 1u) cell(2, y, x0 + 4 * k + j);
            }
        }
    } else {
        for (int i = threadIdx.x; i < TY * TX; i += blockDim.x) {
            const int y = i / TX, x = i - (i / TX) * TX;
            const int64_t g = (int64_t)(ty0 + y) * W + tx0 + x;
            const uint8_t st = Fe[g];
            Foe[g] = st;
            cell(st, y, x);
        }
    }
    a = __reduce_or_sync(0xffffffffu, a);
    nd = __reduce_add_sync(0xffffffffu, nd);
    if ((threadIdx.x & 31) == 0) {
        if (a) atomicOr(&s_act, a);
        if (nd) atomicAdd(&s_burnt, nd);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        act[tix] = (uint16_t)s_act;
        synced[tix] = 1;
        tile_burnt[tix] = s_burnt;
    }
}

// Persistent CTAs take the round's items from the plan: the active tiles
// (stepped) and then the quiet tiles whose interior is copied once to the
// other buffer.
// resident CTAs per SM the register budget is set for, and the work items a
// thread of the fused variant evaluates at once
__host__ __device__ constexpr int tiled_min_blocks(int nt) { return nt == 256 ? 2 : nt == 128 ? 4 : 1; }
__host__ __device__ constexpr int tiled_ilp(int nt) { return nt == 512 ? 4 : 2; }

template <int NT, bool FUSED>
__global__ void __launch_bounds__(NT, tiled_min_blocks(NT))
k_step_tiled(const TileArgs a, const RateConsts Kc) {
    extern __shared__ uint32_t sm[];
    // per step: interior burning, interior burn-outs, interior cells doused by
    // the next step's drop, region burning
    __shared__ int32_t s_cnt[3][4];
    __shared__ int32_t s_d0;
    __shared__ uint32_t s_act;
    __shared__ int32_t s_qn[3];
    __shared__ int s_item;
    __shared__ int s_tma;
    __shared__ alignas(8) uint64_t s_bar;
    __shared__ typename std::conditional<FUSED, RateConsts, int>::type sK_store;
    const RateConsts& sK = *reinterpret_cast<const RateConsts*>(&sK_store);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (FUSED) {
        for (int i = threadIdx.x; i < (int)(sizeof(RateConsts) / 4); i += NT)
            reinterpret_cast<float*>(&sK_store)[i] = reinterpret_cast<const float*>(&Kc)[i];
    }
    const int32_t n_act = a.plan[0], n_copy = a.plan[1];
    const int32_t* act_list = a.plan + 4 + a.N;
    const int32_t* copy_list = act_list + a.n_tiles;
    // only thread 0 uses the barrier: it counts the completed tensor copies
    // and waits for phase parity ph
    uint32_t ph = 0;
    if (threadIdx.x == 0) jwf_mbar_init(&s_bar, 1);
    const int kb = a.kb;
    for (;;) {
    // each thread's earlier shared-memory accesses are ordered before the
    // next tensor copy into the same memory
    jwf_fence_proxy_async();
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(&a.plan[2], 1);
    __syncthreads();
    const int item = s_item;
    if (item >= n_act + n_copy) break;
    const bool is_copy = item >= n_act;
    const int tix = is_copy ? copy_list[item - n_act] : act_list[item];
    const int4 tl = a.tiles[tix];
    const int e = tl.x, tr = tl.y, tc = tl.z;
    const int H = a.H[e], W = a.W[e];
    const int64_t off = a.off[e];
    const int ty0 = tr * kTileRows, tx0 = tc * kTileCols;
    const int TY = min(kTileRows, H - ty0), TX = min(kTileCols, W - tx0);
    const bool use_tma = a.tma_ok != nullptr && a.tma_ok[e] != 0;
    if (is_copy) {
        // no fire within reach: the interior stays as it is; copy it once to
        // the other buffer (cells outside the grid are neither read nor written)
        if (use_tma) {
            if (threadIdx.x == 0) {
                uint8_t* stg = reinterpret_cast<uint8_t*>(sm) + ((128u - (jwf_smem_u32(sm) & 127u)) & 127u);
                jwf_mbar_expect_tx(&s_bar, kTileRows * kTileCols);
                if (!a.diag_no_copy) jwf_tma_load_2d(stg, a.tm_in_tile + e, tx0, ty0, &s_bar);
                int ok = 1;
                if (jwf_mbar_wait_bounded(&s_bar, ph, a.wait_ns)) {
                    jwf_tma_store_2d(a.tm_out_tile + e, tx0, ty0, stg);
                    jwf_bulk_commit();
                    jwf_bulk_wait_all();
                } else {
                    atomicOr(a.status, JWF_DEVERR_TMA);
                    jwf_mbar_wait_bounded(&s_bar, ph, a.wait_ns);      // a late copy lands before the exit
                    ok = 0;
                }
                ph ^= 1u;
                a.synced[tix] = (uint8_t)ok;
                s_tma = ok;
            }
            __syncthreads();
            if (!s_tma) break;          // the barrier's phase is unknown: this CTA stops
        } else {
            for (int i = threadIdx.x; i < TY * TX; i += NT) {
                const int64_t g = off + (int64_t)(ty0 + i / TX) * W + tx0 + i % TX;
                a.Fout[g] = a.Fin[g];
            }
            if (threadIdx.x == 0) a.synced[tix] = 1;
        }
        continue;
    }
    // region: rows [ty0 - kb, ty0 + TY + kb), columns [tx0 - 32, tx0 + TX + 32)
    const int oy = ty0 - kb, ox = tx0 - 32;
    const int RH = TY + 2 * kb;
    const int WW = (TX + 64 + 31) >> 5;
    const WordDiv wd(WW);
    const int pw = (RH + 2) * WW;
    const int words = RH * WW;
    const int nchunks = (words + 31) >> 5;
    uint32_t* B0 = sm;
    uint32_t* B1 = B0 + pw;
    uint32_t* C = B1 + pw;
    uint32_t* D = C + words;
    uint32_t* list = D + words + warp * kWarpScratch;
    uint32_t* ignw = list + kListCap;
    uint32_t* outw = ignw + 32;
    uint32_t* plist = outw + 32;
    // chunk activity flags of the two burning buffers (as in the resident step)
    uint8_t* fl_c = reinterpret_cast<uint8_t*>(D + words + (NT / 32) * kWarpScratch);
    uint8_t* fl_n = fl_c + kTileFlagBytes;
    uint32_t* IG = reinterpret_cast<uint32_t*>(fl_c + 2 * kTileFlagBytes);   // ignitions this step
    uint32_t* OU = IG + kRegionWordsAll;                                      // burn-outs this step
    uint32_t* Q = OU + kRegionWordsAll;
    int* wch = reinterpret_cast<int*>(Q + kQCap) + warp * kRegionChunks;     // chunks dealt to this warp
    const int reach = (WW + 1 + 31) >> 5;
    // the region's bytes are staged where the ignition, burn-out and queue
    // arrays go (they are not used before the steps start)
    uint8_t* stg = reinterpret_cast<uint8_t*>(IG) + ((128u - (jwf_smem_u32(IG) & 127u)) & 127u);
    if (use_tma && threadIdx.x == 0) {
        // region rows [ty0 - kb, ty0 - kb + kBoxRows), columns [tx0 - 32, tx0 + 160):
        // x is a multiple of 32 cells; rows and columns outside the grid read as 0
        jwf_mbar_expect_tx(&s_bar, kBoxRows * kBoxCols);
        if (!a.diag_no_copy) jwf_tma_load_2d(stg, a.tm_region + e, tx0 - 32, ty0 - kb, &s_bar);
    }
    for (int i = threadIdx.x; i < 2 * pw; i += NT) B0[i] = 0u;
    if (threadIdx.x < 3) s_qn[threadIdx.x] = 0;
    if (threadIdx.x < 12) s_cnt[threadIdx.x / 4][threadIdx.x % 4] = 0;
    if (threadIdx.x == 0) {
        s_d0 = 0;
        s_act = 0u;
    }
    ignw[lane] = 0u;
    outw[lane] = 0u;
    if (use_tma && threadIdx.x == 0) s_tma = jwf_mbar_wait_bounded(&s_bar, ph, a.wait_ns) ? 1 : 0;
    __syncthreads();
    if (use_tma && !s_tma) {
        // the copy did not complete: report, let a late copy land, and stop
        // (the barrier's phase is unknown; other CTAs take the remaining tiles)
        if (threadIdx.x == 0) {
            atomicOr(a.status, JWF_DEVERR_TMA);
            jwf_mbar_wait_bounded(&s_bar, ph, a.wait_ns);
        }
        break;
    }
    if (use_tma) ph ^= 1u;
    // load the region (cells outside the grid read as no fuel)
    for (int i = threadIdx.x; i < words; i += NT) {
        const int ry = wd.div(i), w = i - ry * WW;
        const int gy = oy + ry, gx0 = ox + (w << 5);
        uint32_t b = 0, c = 0, dd = 0;
        if (use_tma) {
            const uint4* src = reinterpret_cast<const uint4*>(stg + ry * kBoxCols + (w << 5));
            const uint4 lo = src[0], hi = src[1];
            const uint32_t v8[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                c |= nib_eq(v8[k], 0x01010101u) << (4 * k);
                b |= nib_eq(v8[k], 0x02020202u) << (4 * k);
                dd |= nib_eq(v8[k], 0x03030303u) << (4 * k);
            }
        } else if (gy >= 0 && gy < H) {
            const uint8_t* src = a.Fin + off + (int64_t)gy * W + gx0;
            if (gx0 >= 0 && gx0 + 32 <= W && (reinterpret_cast<uintptr_t>(src) & 15u) == 0) {
                const uint4 lo = __ldg(reinterpret_cast<const uint4*>(src));
                const uint4 hi = __ldg(reinterpret_cast<const uint4*>(src) + 1);
                const uint32_t v8[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    c |= nib_eq(v8[k], 0x01010101u) << (4 * k);
                    b |= nib_eq(v8[k], 0x02020202u) << (4 * k);
                    dd |= nib_eq(v8[k], 0x03030303u) << (4 * k);
                }
            } else {
                for (int j = 0; j < 32; ++j) {
                    const int gx = gx0 + j;
                    if (gx < 0 || gx >= W) continue;
                    const uint32_t st = src[j];
                    b |= (uint32_t)(st == 2) << j;
                    c |= (uint32_t)(st == 1) << j;
                    dd |= (uint32_t)(st == 3) << j;
                }
            }
        }
        B0[(ry + 1) * WW + w] = b;
        C[i] = c;
        D[i] = dd;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < words; i += NT) {
        IG[i] = 0u;
        OU[i] = 0u;
    }
    if (a.drops != nullptr) {
        const int gcx = a.drops[(int64_t)e * 2], gcy = a.drops[(int64_t)e * 2 + 1];
        res_action_rel(RH, WW, B0, D, gcx - ox, gcy - oy, a.R, gcx >= 0 && gcy >= 0);
        __syncthreads();
    } else if (a.mask != nullptr) {
        for (int i = threadIdx.x; i < words; i += NT) {
            const int y = wd.div(i), w = i - y * WW;
            uint32_t* bp = &B0[(y + 1) * WW + w];
            if (*bp == 0u) continue;
            const uint32_t m = region_mask(a.mask, off, oy + y, ox + (w << 5), H, W);
            D[i] |= *bp & m;
            *bp &= ~m;
        }
        __syncthreads();
    }
    // initial chunk flags and burned interior cells (after the round's first drop)
    {
        int nd0 = 0;
        for (int c = threadIdx.x; c < nchunks; c += NT) {
            uint32_t any = 0u;
            const int i1 = min(words, (c + 1) << 5);
            for (int i = c << 5; i < i1; ++i) {
                any |= B0[WW + i];
                const int y = wd.div(i), w = i - y * WW;
                if (y >= kb && y < kb + TY) nd0 += __popc(D[i] & col_bits(w, 32, 32 + TX));
            }
            fl_c[c] = any != 0u;
            fl_n[c] = 0;
        }
        if (nd0) atomicAdd(&s_d0, nd0);
    }
    __syncthreads();
    int32_t dbase = s_d0;
    int32_t t0 = a.t[e];
    const uint32_t ep4 = 4u * (uint32_t)a.episode[e];
    uint32_t* Bc = B0;
    uint32_t* Bn = B1;
    int32_t fin_b = 0, fin_d = 0;
    for (int s = 0; s < kb; ++s) {
        const uint32_t tt = (uint32_t)(t0 + s);
        if (threadIdx.x == 0) {
            s_cnt[(s + 1) % 3][0] = 0;
            s_cnt[(s + 1) % 3][1] = 0;
            s_cnt[(s + 1) % 3][2] = 0;
            s_cnt[(s + 1) % 3][3] = 0;
            s_qn[(s + 1) % 3] = 0;
        }
        const uint32_t* mrow = (a.mask != nullptr && s + 1 < kb) ? a.mask + (int64_t)(s + 1) * a.mask_words : nullptr;
        bool hasn = false;
        int cxn = 0, cyn = 0;
        if (a.drops != nullptr && s + 1 < kb) {
            const int gcx = a.drops[((int64_t)(s + 1) * a.N + e) * 2];
            const int gcy = a.drops[((int64_t)(s + 1) * a.N + e) * 2 + 1];
            hasn = gcx >= 0 && gcy >= 0;
            cxn = gcx - ox;
            cyn = gcy - oy;
        }
        int my_b = 0, my_o = 0, my_x = 0, my_r = 0;
        uint32_t my_pairs = 0, my_blocks = 0, my_burn = 0, my_chunks = 0;
        // phase A: the chunks that can change are dealt to the warps, which queue their work
        // items (one per burning cell; one per compared pair in the fused
        // variant, one per candidate cell in the table variant)
        // (a chunk with no burning cell within reach, whose write buffer holds
        // no burning word, cannot change and is skipped; the needed chunks of
        // a group of 32 are found by one ballot and the k-th goes to warp
        // k mod (warps))
        int n_need = 0;
        for (int g0 = 0; g0 < nchunks; g0 += 32) {
            const int cl = g0 + lane;
            bool nd = false;
            if (cl < nchunks) {
                nd = fl_n[cl] != 0;
                for (int cc = max(cl - reach, 0); cc <= min(cl + reach, nchunks - 1); ++cc) nd |= fl_c[cc] != 0;
            }
            const uint32_t need_m = __ballot_sync(0xffffffffu, nd);
            const int rk = n_need + __popc(need_m & ((1u << lane) - 1u));
            n_need += __popc(need_m);
            for (uint32_t mine = __ballot_sync(0xffffffffu, nd && (rk % (NT / 32)) == warp); mine != 0u;) {
            const int c = g0 + __ffs(mine) - 1;
            mine &= mine - 1u;
            if (lane == 0) wch[my_chunks] = c;
            ++my_chunks;
            const int base = c << 5;
            const int i = base + lane;
            uint32_t burn = 0, cand = 0;
            uint32_t sd[8];
            // rows of the region that can still reach the interior by the
            // round's end: at step s, those within kb - 1 - s rows of it
            // (fire moves one cell a step); the others keep their state
            // (stale, never read by a row that matters)
            const int ry = wd.div(i);
            if (i < words && ry > s && ry < RH - 1 - s) {
                const int w = i - ry * WW;
                const uint32_t* bp = &Bc[WW + i];
                const bool hl = w > 0, hr = w + 1 < WW;
                const uint32_t bc = bp[0], bl = hl ? bp[-1] : 0u, br = hr ? bp[1] : 0u;
                const uint32_t uc = bp[-WW], ul = hl ? bp[-WW - 1] : 0u, ur = hr ? bp[-WW + 1] : 0u;
                const uint32_t dc = bp[WW], dl = hl ? bp[WW - 1] : 0u, dr = hr ? bp[WW + 1] : 0u;
                sd[0] = (bc << 1) | (bl >> 31);
                sd[1] = (dc << 1) | (dl >> 31);
                sd[2] = dc;
                sd[3] = (dc >> 1) | (dr << 31);
                sd[4] = (bc >> 1) | (br << 31);
                sd[5] = (uc >> 1) | (ur << 31);
                sd[6] = uc;
                sd[7] = (uc << 1) | (ul >> 31);
                const uint32_t any = sd[0] | sd[1] | sd[2] | sd[3] | sd[4] | sd[5] | sd[6] | sd[7];
                cand = C[i] & any;
                burn = bc;
            } else {
#pragma unroll
                for (int d = 0; d < 8; ++d) sd[d] = 0u;
            }
            uint32_t np = 0;
#pragma unroll
            for (int d = 0; d < 8; ++d) np += __popc(sd[d] & cand);
            my_pairs += np;
            my_blocks += __popc(cand & (sd[0] | sd[1] | sd[2] | sd[3])) + __popc(cand & (sd[4] | sd[5] | sd[6] | sd[7]));
            my_burn += __popc(burn);
            const int n_items = __popc(burn) + (int)(FUSED ? np : __popc(cand));
            int incl = n_items;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            if (total == 0) continue;
            // one reservation of `total` slots; one that runs past the
            // capacity voids the slots it got and the warp evaluates the
            // chunk itself
            int old = 0;
            if (lane == 0) old = atomicAdd(&s_qn[s % 3], total);
            old = __shfl_sync(0xffffffffu, old, 0);
            const int pos = old + total <= kQCap ? old : -1;
            if (pos < 0) {
                for (int j = old + lane; j < min(kQCap, old + total); j += 32) Q[j] = kTileVoid;
            } else {
                uint32_t* q = Q + pos + (incl - n_items);
                const uint32_t hi = (uint32_t)i << 20;
                for (uint32_t m = burn; m != 0u; m &= m - 1u) *q++ = hi | ((uint32_t)(__ffs(m) - 1) << 15);
                if (FUSED) {
#pragma unroll
                    for (int d = 0; d < 8; ++d)
                        for (uint32_t m = sd[d] & cand; m != 0u; m &= m - 1u)
                            *q++ = hi | ((uint32_t)(__ffs(m) - 1) << 15) | (1u << 14) | (uint32_t)d;
                } else {
                    for (uint32_t m = cand; m != 0u; m &= m - 1u) {
                        const int j = __ffs(m) - 1;
                        uint32_t dm = 0;
#pragma unroll
                        for (int d = 0; d < 8; ++d) dm |= ((sd[d] >> j) & 1u) << d;
                        *q++ = hi | ((uint32_t)j << 15) | (1u << 14) | dm;
                    }
                }
                continue;
            }
            // the queue is full: this warp evaluates the chunk itself
            uint32_t* ignw_c = IG + base;
            uint32_t* outw_c = OU + base;
            const uint32_t act = cand | burn;
            const int n_act = __popc(act);
            int inca = n_act;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, inca, o);
                if (lane >= o) inca += v;
            }
            const int tot_a = __shfl_sync(0xffffffffu, inca, 31);
            const int excl = inca - n_act;
            for (int pass = 0; pass < tot_a; pass += kListCap) {
                uint32_t rem = act;
                int idx = excl;
                while (rem != 0u) {
                    const int j = __ffs(rem) - 1;
                    rem &= rem - 1u;
                    if (idx >= pass && idx < pass + kListCap) {
                        uint32_t item = ((uint32_t)lane << 5) | (uint32_t)j;
                        if ((cand >> j) & 1u) {
                            uint32_t dm = 0;
#pragma unroll
                            for (int d = 0; d < 8; ++d) dm |= ((sd[d] >> j) & 1u) << d;
                            item |= (dm << 10) | (1u << 18);
                        }
                        list[idx - pass] = item;
                    }
                    ++idx;
                }
                __syncwarp();
                const int n_pass = min(kListCap, tot_a - pass);
                for (int it = lane; it < n_pass; it += 32) {
                    const uint32_t item = list[it];
                    const int ol = (int)(item >> 5) & 31;
                    const int j = (int)item & 31;
                    const int ii = base + ol;
                    const int ry = wd.div(ii);
                    const int gy = oy + ry, gx = ox + ((ii - ry * WW) << 5) + j;
                    const uint32_t cell = (uint32_t)(gy * W + gx);
                    if (item & (1u << 18)) {
                        if (!FUSED && ignites(a, e, off, cell, (item >> 10) & 0xFFu, tt, ep4))
                            atomicOr(&ignw_c[ol], 1u << j);
                    } else {
                        const uint4 u = jwf_philox(make_uint4(cell, tt, (uint32_t)e, ep4 + 2u), a.key0, a.key1);
                        if (!(jwf_u24(u.x) < a.p_continue)) atomicOr(&outw_c[ol], 1u << j);
                    }
                }
                if (FUSED) {
                    for (int it0 = 0; it0 < n_pass; it0 += 32)
                        fused_pairs(a, sK, list, plist, ignw_c, it0, n_pass, base, e, off, W, WW, oy, ox, tt, ep4,
                                    lane);
                }
                __syncwarp();
            }
            }
        }
        __syncthreads();
        // phase B: every thread of the CTA evaluates queued items (the fused
        // variant several at a time)
        if (FUSED) {
            constexpr int ILP = tiled_ilp(NT);
            const int qn = min(s_qn[s % 3], kQCap);
            for (int q0 = threadIdx.x; q0 < qn; q0 += NT * ILP) {
                int yy[ILP], xx[ILP], kind[ILP], dd[ILP], iis[ILP], js[ILP];
#pragma unroll
                for (int k = 0; k < ILP; ++k) {
                    const int q = q0 + k * NT;
                    const uint32_t it = q < qn ? Q[q] : kTileVoid;
                    if (it == kTileVoid) {
                        // no item: the tile's first cell, nothing loaded for it
                        yy[k] = ty0;
                        xx[k] = tx0;
                        kind[k] = 0;
                        dd[k] = 0;
                        iis[k] = 0;
                        js[k] = 0;
                        continue;
                    }
                    const int ii = (int)(it >> 20), j = (int)(it >> 15) & 31;
                    const int ry = wd.div(ii);
                    yy[k] = oy + ry;
                    xx[k] = ox + ((ii - ry * WW) << 5) + j;
                    kind[k] = (it & (1u << 14)) ? 2 : 1;
                    dd[k] = (int)(it & 7u);
                    iis[k] = ii;
                    js[k] = j;
                }
                bool below[ILP];
                eval_items<ILP>(a, sK, e, off, W, yy, xx, kind, dd, tt, ep4, below);
#pragma unroll
                for (int k = 0; k < ILP; ++k) {
                    if (kind[k] == 2 && below[k]) atomicOr(&IG[iis[k]], 1u << js[k]);
                    if (kind[k] == 1 && !below[k]) atomicOr(&OU[iis[k]], 1u << js[k]);
                }
            }
        } else {
            const int qn = min(s_qn[s % 3], kQCap);
            for (int q = threadIdx.x; q < qn; q += NT) {
                const uint32_t it = Q[q];
                if (it == kTileVoid) continue;
                const int ii = (int)(it >> 20), j = (int)(it >> 15) & 31;
                const int ry = wd.div(ii);
                const int gy = oy + ry, gx = ox + ((ii - ry * WW) << 5) + j;
                const uint32_t cell = (uint32_t)(gy * W + gx);
                if (!(it & (1u << 14))) {
                    const uint4 u = jwf_philox(make_uint4(cell, tt, (uint32_t)e, ep4 + 2u), a.key0, a.key1);
                    if (!(jwf_u24(u.x) < a.p_continue)) atomicOr(&OU[ii], 1u << j);
                } else if (FUSED) {
                    if (pair_ignites(a, sK, e, off, W, gy, gx, (int)(it & 7u), tt, ep4)) atomicOr(&IG[ii], 1u << j);
                } else {
                    if (ignites(a, e, off, cell, it & 0xFFu, tt, ep4)) atomicOr(&IG[ii], 1u << j);
                }
            }
        }
        __syncthreads();
        // phase C: each warp writes back the chunks dealt to it
        for (int k = 0; k < (int)my_chunks; ++k) {
            const int c = wch[k];
            const int i = (c << 5) + lane;
            uint32_t nbw = 0u;
            if (i < words) {
                const int y = wd.div(i), w = i - y * WW;
                const uint32_t burn = Bc[WW + i];
                const uint32_t ig = IG[i], ou = OU[i];
                uint32_t nb = (burn & ~ou) | ig;
                const uint32_t im = (y >= kb && y < kb + TY) ? col_bits(w, 32, 32 + TX) : 0u;
                my_r += __popc(nb);
                my_b += __popc(nb & im);
                my_o += __popc(ou & im);
                const uint32_t m = mrow != nullptr ? region_mask(mrow, off, oy + y, ox + (w << 5), H, W)
                                                   : drop_bits_rel(y, w, cxn, cyn, a.R, hasn);
                const uint32_t doused = nb & m;
                my_x += __popc(doused & im);
                nb &= ~m;
                Bn[WW + i] = nb;
                D[i] |= ou | doused;
                C[i] &= ~ig;
                IG[i] = 0u;
                OU[i] = 0u;
                nbw = nb;
            }
            const uint32_t any_nb = __ballot_sync(0xffffffffu, nbw != 0u);
            if (lane == 0) fl_n[c] = any_nb != 0u;
        }
        if (a.counts != nullptr && my_chunks) {
            my_pairs = __reduce_add_sync(0xffffffffu, my_pairs);
            my_blocks = __reduce_add_sync(0xffffffffu, my_blocks);
            my_burn = __reduce_add_sync(0xffffffffu, my_burn);
            if (lane == 0) {
                atomicAdd(&a.counts[0], (unsigned long long)my_pairs);
                atomicAdd(&a.counts[1], (unsigned long long)my_blocks);
                atomicAdd(&a.counts[2], (unsigned long long)my_burn);
                atomicAdd(&a.counts[3], 32ull * my_chunks);
            }
        }
        if (my_chunks) {
            my_b = __reduce_add_sync(0xffffffffu, my_b);
            my_o = __reduce_add_sync(0xffffffffu, my_o);
            my_x = __reduce_add_sync(0xffffffffu, my_x);
            my_r = __reduce_add_sync(0xffffffffu, my_r);
            if (lane == 0) {
                if (my_b) atomicAdd(&s_cnt[s % 3][0], my_b);
                if (my_o) atomicAdd(&s_cnt[s % 3][1], my_o);
                if (my_x) atomicAdd(&s_cnt[s % 3][2], my_x);
                if (my_r) atomicAdd(&s_cnt[s % 3][3], my_r);
            }
        }
        __syncthreads();
        fin_b = s_cnt[s % 3][0];
        fin_d = dbase + s_cnt[s % 3][1];          // burned after the step
        dbase = fin_d + s_cnt[s % 3][2];          // and after the next drop
        const int32_t nr = s_cnt[s % 3][3];
        if (threadIdx.x == 0) {
            if (fin_b) atomicAdd(&a.cnt[((int64_t)s * 2) * a.N + e], fin_b);
            if (fin_d) atomicAdd(&a.cnt[((int64_t)s * 2 + 1) * a.N + e], fin_d);
        }
        uint32_t* tmp = Bc;
        Bc = Bn;
        Bn = tmp;
        uint8_t* ftmp = fl_c;
        fl_c = fl_n;
        fl_n = ftmp;
        if (nr == 0) {
            // no fire left in the region: the remaining steps change nothing
            for (int s2 = s + 1 + (int)threadIdx.x; s2 < kb; s2 += NT)
                if (fin_d) atomicAdd(&a.cnt[((int64_t)s2 * 2 + 1) * a.N + e], fin_d);
            break;
        }
    }
    __syncthreads();
    // write the interior back to the other buffer
    const int iwords = (TX + 31) >> 5;
    for (int i = threadIdx.x; i < TY * iwords; i += NT) {
        const int ry = kb + i / iwords, w = 1 + i % iwords;
        const int gy = oy + ry, gx0 = ox + (w << 5);
        uint8_t* dst = a.Fout + off + (int64_t)gy * W + gx0;
        const uint32_t b = Bc[(ry + 1) * WW + w], c = C[ry * WW + w], dd = D[ry * WW + w];
        const int n = min(32, tx0 + TX - gx0);
        if (n == 32 && (reinterpret_cast<uintptr_t>(dst) & 15u) == 0) {
            uint32_t v8[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int sh = 4 * k;
                v8[k] = nib_spread((c >> sh) & 0xFu) + 2u * nib_spread((b >> sh) & 0xFu) +
                        3u * nib_spread((dd >> sh) & 0xFu);
            }
            reinterpret_cast<uint4*>(dst)[0] = make_uint4(v8[0], v8[1], v8[2], v8[3]);
            reinterpret_cast<uint4*>(dst)[1] = make_uint4(v8[4], v8[5], v8[6], v8[7]);
        } else {
            for (int j = 0; j < n; ++j)
                dst[j] = (uint8_t)(((c >> j) & 1u) + ((b >> j) & 1u) * 2u + ((dd >> j) & 1u) * 3u);
        }
    }
    // where the burning interior cells are, for the next round's activity
    uint32_t act = 0u;
    if (fin_b > 0) {
        const int band = kMaxRound;
        for (int i = threadIdx.x; i < TY * iwords; i += NT) {
            const int ry = kb + i / iwords, w = 1 + i % iwords;
            const uint32_t b = Bc[(ry + 1) * WW + w] & col_bits(w, 32, 32 + TX);
            if (b == 0u) continue;
            act |= kActAny;
            const bool n = ry - kb < band, so = kb + TY - 1 - ry < band;
            const bool wb = (b & col_bits(w, 32, 32 + band)) != 0u;
            const bool eb = (b & col_bits(w, max(32, 32 + TX - band), 32 + TX)) != 0u;
            if (n) act |= kActN;
            if (so) act |= kActS;
            if (wb) act |= kActW;
            if (eb) act |= kActE;
            if (n && wb) act |= kActNW;
            if (n && eb) act |= kActNE;
            if (so && wb) act |= kActSW;
            if (so && eb) act |= kActSE;
        }
        act = __reduce_or_sync(0xffffffffu, act);
        if (lane == 0 && act != 0u) atomicOr(&s_act, act);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        a.tile_burnt[tix] = fin_d;
        a.act_out[tix] = (uint16_t)s_act;
        a.synced[tix] = 0;
    }
    }
}

// After a round: per-step outputs (burned = the active tiles' per-step
// counts + the quiet tiles' cells), done flags and t += kb, one thread per
// env; the plan's header and per-env sums are cleared for the next round.
struct FinalArgs {
    int32_t N, kb;
    const int32_t* cnt;
    int32_t* plan;
    int32_t* t;
    int32_t t_max;
    int32_t* burning;
    int32_t* burnt;
    uint8_t* done;
};

__device__ __forceinline__ void round_finalize_part(const FinalArgs& f, int e) {
    const int32_t N = f.N, kb = f.kb, t_max = f.t_max;
    const int32_t* __restrict__ cnt = f.cnt;
    int32_t* __restrict__ plan = f.plan;
    int32_t* __restrict__ t = f.t;
    int32_t* __restrict__ burning = f.burning;
    int32_t* __restrict__ burnt = f.burnt;
    uint8_t* __restrict__ done = f.done;
    if (e == 0) {
        plan[0] = 0;
        plan[1] = 0;
        plan[2] = 0;
    }
    if (e >= N) return;
    const int32_t quiet = plan[4 + e];
    plan[4 + e] = 0;
    const int32_t t0 = t[e];
    for (int s = 0; s < kb; ++s) {
        const int32_t nb = cnt[((int64_t)s * 2) * N + e], nd = cnt[((int64_t)s * 2 + 1) * N + e] + quiet;
        const int64_t o = (int64_t)s * N + e;
        if (burning) burning[o] = nb;
        if (burnt) burnt[o] = nd;
        if (done) done[o] = (nb == 0 || (t_max > 0 && t0 + s + 1 >= t_max)) ? 1 : 0;
    }
    t[e] = t0 + kb;
}

__global__ void k_round_finalize(const FinalArgs f) { round_finalize_part(f, blockIdx.x * blockDim.x + threadIdx.x); }

// A round's close and the next round's plan in one launch: the two rounds'
// plans and count scratch are separate buffers, so the parts share no data.
__global__ void __launch_bounds__(256) k_round_next(const FinalArgs f, const PlanArgs p) {
    const int64_t tix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tix < f.N) round_finalize_part(f, (int)tix);
    tile_plan_part(p, tix);
}

constexpr int kMaxDev = 64;

// One persistent CTA per resident slot (never more than there are tiles);
// the attribute and occupancy queries run once per device.
template <int NT, bool FUSED>
cudaError_t launch_tiled_t(const jwf_ctx* c, const TileArgs& a, const RateConsts& K, cudaStream_t s) {
    static int per_sm[kMaxDev] = {};
    const size_t smem = tiled_smem_bytes(NT);
    const int dev = c->device;
    if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
    if (per_sm[dev] == 0) {
        cudaError_t err = cudaFuncSetAttribute(k_step_tiled<NT, FUSED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem);
        if (err != cudaSuccess) return err;
        int n = 0;
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_tiled<NT, FUSED>, NT, smem);
        if (err != cudaSuccess) return err;
        if (n < 1) return cudaErrorInvalidConfiguration;
        per_sm[dev] = n;
    }
    int64_t grid = (int64_t)per_sm[dev] * c->num_sms;
    if (grid > c->n_tiles4) grid = c->n_tiles4;
    k_step_tiled<NT, FUSED><<<(unsigned)grid, NT, smem, s>>>(a, K);
    return cudaGetLastError();
}
}  // namespace

void jwf_rate_consts(const jwf_ctx* c, RateConsts* K);

int jwf_tile_rows() { return kTileRows; }
int jwf_tile_cols() { return kTileCols; }

cudaError_t jwf_launch_step_tiled(jwf_ctx* c, int32_t k, const int32_t* drops, const uint32_t* masks,
                                  int32_t* burning, int32_t* burnt, uint8_t* done, bool fused, cudaStream_t s) {
    const int64_t mw = jwf_mask_row_words(c->cells);
    cudaError_t err;
    if (!c->tiles_valid) {
        // the state changed outside the tiled path: each tile's activity and
        // burned cells from the current state
        k_tile_act_init<<<(unsigned)c->n_tiles4, 256, 0, s>>>(c->d_tiles4, c->d_H, c->d_W, c->d_off,
                                                             c->d_state[c->cur], c->d_state[c->cur ^ 1],
                                                             c->d_tact[c->tact_cur],
                                                             c->d_tsync, c->d_tburnt);
        err = cudaGetLastError();
        if (err != cudaSuccess) return err;
        c->tiles_valid = true;
    }
    RateConsts K;
    if (fused)
        jwf_rate_consts(c, &K);
    else
        K = RateConsts{};
    int32_t rs = (c->round_steps >= 1 && c->round_steps <= kMaxRound) ? c->round_steps : kMaxRound;
    if (c->hist != nullptr) rs = 1;     // recording: the state after every step
    // rounds alternate between two plans and two count scratch buffers: the
    // launch that closes a round also plans the next one
    const int64_t plan_words = 4 + (int64_t)c->N + 2 * c->n_tiles4;
    const int64_t cnt_words = (int64_t)kMaxRound * 2 * c->N;
    const unsigned plan_blocks = (unsigned)((c->n_tiles4 + 255) / 256);
    auto plan_args = [&](int buf, int32_t kb_r) {
        PlanArgs p;
        p.n_tiles = c->n_tiles4;
        p.tiles = c->d_tiles4;
        p.env_tiles = c->d_env_tiles;
        // the round reads the activity the previous round left (tact_cur)
        p.act_in = c->d_tact[c->tact_cur];
        p.act_out = c->d_tact[c->tact_cur ^ 1];
        p.synced = c->d_tsync;
        p.tile_burnt = c->d_tburnt;
        p.N = c->N;
        p.plan = c->d_tplan + buf * plan_words;
        p.cnt = c->d_tcnt + buf * cnt_words;
        p.n_cnt = (int64_t)kb_r * 2 * c->N;
        return p;
    };
    if (k > 0) {
        // the first round's plan: active tiles, quiet tiles to copy, the quiet
        // tiles' burned cells per env (and the round's count scratch zeroed)
        k_tile_plan<<<plan_blocks, 256, 0, s>>>(plan_args(c->tplan_cur, k < rs ? k : rs));
        err = cudaGetLastError();
        if (err != cudaSuccess) return err;
    }
    for (int32_t s0 = 0; s0 < k; s0 += rs) {
        const int32_t kb = (k - s0) < rs ? (k - s0) : rs;
        const int pb = c->tplan_cur;
        TileArgs a;
        a.H = c->d_H;
        a.W = c->d_W;
        a.off = c->d_off;
        a.tiles = c->d_tiles4;
        a.env_tiles = c->d_env_tiles;
        a.N = c->N;
        a.Fin = c->d_state[c->cur];
        a.Fout = c->d_state[c->cur ^ 1];
        a.q = c->d_q;
        a.cls = c->t_cls;
        a.dem = c->t_dem;
        a.wexp = c->wser_n > 0 ? c->d_wser : c->d_wexp;
        a.wser_n = c->wser_n;
        a.drops = drops ? drops + (int64_t)s0 * c->N * 2 : nullptr;
        a.mask = masks ? masks + (int64_t)s0 * mw : nullptr;
        a.mask_words = mw;
        a.t = c->d_t;
        a.episode = c->d_episode;
        a.cnt = c->d_tcnt + pb * cnt_words;
        a.act_in = c->d_tact[c->tact_cur];
        a.act_out = c->d_tact[c->tact_cur ^ 1];
        a.synced = c->d_tsync;
        a.tile_burnt = c->d_tburnt;
        a.counts = c->d_pairs;
        const int bi = c->cur, bo = c->cur ^ 1;
        a.tm_region = c->tma && c->use_tma ? c->d_tmaps + (size_t)(2 * bi) * c->N : nullptr;
        a.tm_in_tile = c->tma && c->use_tma ? c->d_tmaps + (size_t)(2 * bi + 1) * c->N : nullptr;
        a.tm_out_tile = c->tma && c->use_tma ? c->d_tmaps + (size_t)(2 * bo + 1) * c->N : nullptr;
        a.tma_ok = c->tma && c->use_tma ? c->d_tma_ok : nullptr;
        a.status = c->d_status;
        a.wait_ns = c->tma_wait_ns;
        a.diag_no_copy = c->tma_diag_no_copy ? 1 : 0;
        a.plan = c->d_tplan + pb * plan_words;
        a.n_tiles = c->n_tiles4;
        a.kb = kb;
        a.R = c->drop_radius;
        a.key0 = (uint32_t)(c->seed & 0xffffffffu);
        a.key1 = (uint32_t)(c->seed >> 32);
        a.p_continue = c->P.p_continue;
        const int nt = c->threads_per_env;
        if (nt == 128)
            err = fused ? launch_tiled_t<128, true>(c, a, K, s) : launch_tiled_t<128, false>(c, a, K, s);
        else if (nt == 512)
            err = fused ? launch_tiled_t<512, true>(c, a, K, s) : launch_tiled_t<512, false>(c, a, K, s);
        else
            err = fused ? launch_tiled_t<256, true>(c, a, K, s) : launch_tiled_t<256, false>(c, a, K, s);
        if (err != cudaSuccess) return err;
        const int64_t o = (int64_t)s0 * c->N;
        FinalArgs f;
        f.N = c->N;
        f.kb = kb;
        f.cnt = c->d_tcnt + pb * cnt_words;
        f.plan = c->d_tplan + pb * plan_words;
        f.t = c->d_t;
        f.t_max = c->t_max;
        f.burning = burning ? burning + o : nullptr;
        f.burnt = burnt ? burnt + o : nullptr;
        f.done = done ? done + o : nullptr;
        const int32_t s1 = s0 + kb;
        c->cur ^= 1;
        c->tact_cur ^= 1;
        c->tplan_cur ^= 1;
        if (s1 < k) {
            // close this round and plan the next in one launch
            k_round_next<<<plan_blocks, 256, 0, s>>>(f, plan_args(c->tplan_cur, (k - s1) < rs ? (k - s1) : rs));
        } else {
            k_round_finalize<<<(c->N + 255) / 256, 256, 0, s>>>(f);
        }
        err = cudaGetLastError();
        if (err != cudaSuccess) return err;
        if (c->hist != nullptr) {
            err = jwf_record_row(c, s0, s);
            if (err != cudaSuccess) return err;
        }
    }
    return cudaSuccess;
}

// Tensor maps of the tiled step: per state buffer b and env e, a map with the
// region box (kBoxCols x kBoxRows) at d_tmaps[(2b) N + e] and one with the tile
// box (kTileCols x kTileRows) at d_tmaps[(2b + 1) N + e].  An env qualifies when
// its first cell and its row pitch (W bytes) are multiples of 16 bytes, as
// the tensor copy requires.
cudaError_t jwf_build_tile_maps(jwf_ctx* c) {
    c->tma = false;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || fn == nullptr) {
        cudaGetLastError();
        return cudaSuccess;     // no encoder: the plain loads serve every env
    }
    using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    const Encode encode = reinterpret_cast<Encode>(fn);
    static_assert(sizeof(CUtensorMap) == sizeof(JwfTmap), "tensor map size");
    const int N = c->N;
    std::vector<JwfTmap> maps((size_t)4 * N);
    std::vector<uint8_t> ok(N, 0);
    bool any = false;
    for (int e = 0; e < N; ++e) {
        const int64_t W = c->W[e], H = c->H[e];
        if ((c->off[e] & 15) != 0 || (W & 15) != 0) continue;
        bool good = true;
        for (int b = 0; b < 2 && good; ++b) {
            for (int kind = 0; kind < 2 && good; ++kind) {
                const cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)H};
                const cuuint64_t strides[1] = {(cuuint64_t)W};
                const cuuint32_t box[2] = {(cuuint32_t)(kind == 0 ? kBoxCols : kTileCols),
                                           (cuuint32_t)(kind == 0 ? kBoxRows : kTileRows)};
                const cuuint32_t estr[2] = {1, 1};
                CUtensorMap* m = reinterpret_cast<CUtensorMap*>(&maps[(size_t)(2 * b + kind) * N + e]);
                good = encode(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, c->d_state[b] + c->off[e], dims, strides, box,
                              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
            }
        }
        ok[e] = good ? 1 : 0;
        any = any || good;
    }
    if (!any) return cudaSuccess;
    cudaError_t err = cudaMalloc(reinterpret_cast<void**>(&c->d_tmaps), maps.size() * sizeof(JwfTmap));
    if (err == cudaSuccess) err = cudaMalloc(reinterpret_cast<void**>(&c->d_tma_ok), (size_t)N);
    if (err == cudaSuccess)
        err = cudaMemcpy(c->d_tmaps, maps.data(), maps.size() * sizeof(JwfTmap), cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemcpy(c->d_tma_ok, ok.data(), (size_t)N, cudaMemcpyHostToDevice);
    if (err == cudaSuccess) c->tma = true;
    return err;
}

