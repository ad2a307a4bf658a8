// k_resident.cu -- the shared-memory-resident discrete step (Section 3
// "Stochastic update", tanker action of Section 4) running k steps per launch.
//
// Persistent CTAs pull whole envs from a work queue (largest first) and keep
// each env in shared memory as bit planes, 32 cells per word: burning B
// (double-buffered, one zero row above and below), can-burn C and burned D.
// One step has three phases separated by barriers:
//   A. the 32-word chunks that can change are found by one ballot per 32
//      chunks and dealt to the warps by rank; for each, a warp finds, one
//      word a lane, the can-burn cells with a burning neighbour and the
//      burning cells (eight shifted ORs of the burning plane); the work items
//      (remain-burning draws, compared (target, source) pairs) go to a
//      block-wide queue in shared memory (one atomicAdd reservation per
//      chunk), and the candidates' terrain rows are prefetched for B;
//   B. all threads of the CTA evaluate the queued items (one Philox block an
//      item; a pair's ignition probability in plain float with a proven
//      error bound, the double-float rate only for draws within it) and set
//      ignition and burn-out bits;
//   C. the dealt chunks are written back (new burning plane, the next
//      step's tanker drop, counts).
// A launch may be split after a few steps (k_reorder between the parts) so
// that the envs with the largest fires start the rest first.
// For grids larger than shared memory, k_step_tiled (k_tiled.cu) steps tiles
// with a halo (temporal blocking).
// The ignition probability of a compared (target, source) pair is read from
// the q table or, in the fused variant, evaluated on the spot with the same
// rate code as the table kernel (rate_model.cuh), so both variants draw the
// same numbers against the same probabilities.  An env whose fire is out
// stops early; with auto-reset it restarts from its initial state instead.
#include <type_traits>

#include "bitplane.cuh"

namespace {

constexpr int kResQCap = 1024;     // block-wide work items per step (resident step)
constexpr uint32_t kResVoid = 0xffffffffu;   // a voided queue slot (real items have bits 8..11 clear)

struct ResArgs {
    const int32_t* H;
    const int32_t* W;
    const int64_t* off;
    const int32_t* order;       // envs of this launch's queue, largest first
    int32_t nq;                 // length of the queue
    int32_t N;                  // envs in the context (row length of drops and outputs)
    uint8_t* F;                 // in/out (in place: one CTA per env)
    const uint8_t* F0;
    const float* q;             // table variant
    const uint8_t* cls;         // fused variant: landcover, elevation, wind exponent
    const float* dem;
    const float2* wexp;         // [N][8] (hi, lo), or [wser_n][N][8] for a wind series
    int32_t wser_n;             // steps of the wind series (0: static wind)
    const int32_t* drops;       // [k][N][2] or null
    const uint32_t* mask;       // [k][mask_words] bit rows of the steps' action masks, or null
    int64_t mask_words;
    int32_t* t;
    int32_t* episode;
    int32_t* out_burning;       // [k][N] or null
    int32_t* out_burnt;
    uint8_t* out_done;
    uint32_t* queue;            // [0] cursor, [1] CTAs finished
    int32_t* last_burning;      // [N] burning cells after the launch's last step, or null
    uint8_t* history;           // [k] rows: the state after each step, or null
    int64_t cells;              // cells of the context
    int64_t hist_stride;        // bytes between history rows
    int32_t hist_packed;        // rows are 2-bit packed (else one byte a cell)
    int32_t packed_aligned;     // every env starts on a 32-cell boundary and W % 32 == 0
    unsigned long long* counts; // optional [4]: pairs compared, candidate Philox blocks,
                                // burning-cell draws, bit-plane word-steps scanned
    int32_t k;
    int32_t t_max;
    int32_t R;
    int32_t auto_reset;
    uint32_t key0, key1;
    float p_continue;
};

// words of dynamic shared memory for the planes of an H x W env
__host__ __device__ __forceinline__ int res_plane_words(int H, int W) {
    const int WW = (W + 31) >> 5;
    return 2 * (H + 2) * WW + 2 * H * WW;
}

// Scalars of the threads that step one env, at the start of its shared
// region.
struct ResEnvShared {
    int32_t env;
    int32_t cnt[3][3];      // burning, new burn-outs, doused (per step, three steps in flight)
    int32_t qn[3];          // queued work items (per step)
    int32_t ncl[3];         // chunks that can change (per step)
    int32_t burnt;
    int32_t dous;           // cells doused by a drop applied at a step's start
    int32_t drop[2];        // the next step's drop centre (x, y), -1 for none
    int32_t burnt_now;      // burned cells after the last step and the next drop (thread 0)
    int32_t last_burnt;     // burned cells after the last step
    int32_t last_nb;        // burning cells after the last step
    int32_t pad;
};
constexpr int kEnvScalarWords = (int)(sizeof(ResEnvShared) / 4);

// words of an env's region: its scalars, the planes, two chunk-flag byte
// arrays, the dealt-chunk list and the work queue
__host__ __device__ __forceinline__ int res_region_words(int H, int W) {
    const int nchunks = (H * ((W + 31) >> 5) + 31) >> 5;
    return kEnvScalarWords + res_plane_words(H, W) + 2 * ((nchunks + 3) >> 2) + nchunks + kResQCap;
}


// Load env into planes: one word (32 cells) per thread iteration.
__device__ void res_load(const uint8_t* __restrict__ Fe, int H, int W, int WW, bool vec,
                         uint32_t* Bp, uint32_t* C, uint32_t* D, int tid, int nth) {
    const int words = H * WW;
    const WordDiv wd(WW);
    for (int i = tid; i < words; i += nth) {
        const int y = wd.div(i), w = i - y * WW;
        const int x0 = w << 5;
        const uint8_t* src = Fe + (int64_t)y * W + x0;
        uint32_t b = 0, c = 0, dd = 0;
        if (vec) {
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
            const int n = min(32, W - x0);
            for (int j = 0; j < n; ++j) {
                const uint32_t s = src[j];
                b |= (uint32_t)(s == 2) << j;
                c |= (uint32_t)(s == 1) << j;
                dd |= (uint32_t)(s == 3) << j;
            }
        }
        Bp[(y + 1) * WW + w] = b;
        C[i] = c;
        D[i] = dd;
    }
}

__device__ void res_store(uint8_t* __restrict__ Fe, int H, int W, int WW, bool vec,
                          const uint32_t* Bp, const uint32_t* C, const uint32_t* D, int tid, int nth) {
    const int words = H * WW;
    const WordDiv wd(WW);
    for (int i = tid; i < words; i += nth) {
        const int y = wd.div(i), w = i - y * WW;
        const int x0 = w << 5;
        uint8_t* dst = Fe + (int64_t)y * W + x0;
        const uint32_t b = Bp[(y + 1) * WW + w], c = C[i], dd = D[i];
        if (vec) {
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
            const int n = min(32, W - x0);
            for (int j = 0; j < n; ++j)
                dst[j] = (uint8_t)(((c >> j) & 1u) + ((b >> j) & 1u) * 2u + ((dd >> j) & 1u) * 3u);
        }
    }
}

// bit j of v -> bit 2j of the result
__device__ __forceinline__ uint64_t spread_bits(uint32_t v) {
    uint64_t x = v;
    x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
    x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
    x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
    x = (x | (x << 2)) & 0x3333333333333333ull;
    return (x | (x << 1)) & 0x5555555555555555ull;
}

// The env's state as 2-bit codes into a packed row P (cell g of the context
// at bits 2g, 2g + 1 of the row; the env's first cell is g = off).  With
// `aligned` every word of 32 cells owns 8 whole bytes (plain stores);
// otherwise words share bytes with their neighbours and OR their bits into a
// row the caller zeroed.
__device__ void res_store2(uint32_t* __restrict__ P, int64_t off, int H, int W, int WW, bool aligned,
                           const uint32_t* Bp, const uint32_t* C, const uint32_t* D, int tid, int nth) {
    const int words = H * WW;
    const WordDiv wd(WW);
    for (int i = tid; i < words; i += nth) {
        const int y = wd.div(i), w = i - y * WW;
        const int x0 = w << 5;
        const int n = min(32, W - x0);
        const uint32_t m = n == 32 ? 0xffffffffu : ((1u << n) - 1u);
        const uint32_t b = Bp[(y + 1) * WW + w], dd = D[i];
        // code = 1 can burn, 2 burning, 3 burned: low bit C|D, high bit B|D
        const uint64_t code = spread_bits((C[i] | dd) & m) | (spread_bits((b | dd) & m) << 1);
        const int64_t g0 = off + (int64_t)y * W + x0;
        if (aligned) {
            reinterpret_cast<uint2*>(P)[g0 >> 5] = make_uint2((uint32_t)code, (uint32_t)(code >> 32));
        } else {
            const int64_t bit = 2 * g0;
            uint32_t* q = P + (bit >> 5);
            const int o = (int)(bit & 31);
            const uint32_t w0 = (uint32_t)(code << o);
            const uint32_t w1 = o ? (uint32_t)(code >> (32 - o)) : (uint32_t)(code >> 32);
            const uint32_t w2 = o ? (uint32_t)(code >> (64 - o)) : 0u;
            if (w0) atomicOr(q, w0);
            if (w1) atomicOr(q + 1, w1);
            if (w2) atomicOr(q + 2, w2);
        }
    }
}

// history row `row` of the env: one byte a cell, or 2-bit packed
__device__ __forceinline__ void res_record(const ResArgs& a, int64_t row, int64_t off, int H, int W, int WW,
                                           bool vec, const uint32_t* Bp, const uint32_t* C, const uint32_t* D,
                                           int tid, int nth) {
    const int64_t ho = row * a.hist_stride;
    if (a.hist_packed)
        res_store2(reinterpret_cast<uint32_t*>(a.history + ho), off, H, W, WW, a.packed_aligned != 0, Bp, C, D,
                   tid, nth);
    else
        res_store(a.history + ho + off, H, W, WW, vec && (ho & 15) == 0, Bp, C, D, tid, nth);
}

// Bits of word w (cells 32w .. 32w+31) of row y covered by a drop of radius R
// at (cx, cy), clipped to the grid; 0 for no drop.
__device__ __forceinline__ uint32_t drop_bits(int y, int w, int W, int cx, int cy, int R) {
    if (cx < 0 || cy < 0 || abs(y - cy) > R) return 0u;
    const int lo = max(max(cx - R, 0) - (w << 5), 0);
    const int hi = min(min(cx + R, W - 1) - (w << 5), 31);
    if (lo > hi) return 0u;
    const uint32_t span = (hi - lo == 31) ? 0xffffffffu : ((1u << (hi - lo + 1)) - 1u);
    return span << lo;
}

// Apply a drop to the planes (burning under it -> burned), all threads; adds
// the number of doused cells to *count when count is not null.
__device__ void res_action(int H, int W, int WW, uint32_t* Bp, uint32_t* D, int cx, int cy, int R, int tid,
                           int nth, int* count = nullptr) {
    if (cx < 0 || cy < 0) return;
    const int y0 = max(cy - R, 0), y1 = min(cy + R, H - 1);
    if (y0 > y1) return;
    const int w0 = max(cx - R, 0) >> 5, w1 = min(cx + R, W - 1) >> 5;
    const int nw = w1 - w0 + 1;
    const int total = (y1 - y0 + 1) * nw;
    for (int j = tid; j < total; j += nth) {
        const int y = y0 + j / nw, w = w0 + j % nw;
        const uint32_t m = drop_bits(y, w, W, cx, cy, R);
        uint32_t* bp = &Bp[(y + 1) * WW + w];
        const uint32_t doused = *bp & m;
        *bp &= ~m;
        D[y * WW + w] |= doused;
        if (count != nullptr && doused != 0u) atomicAdd(count, __popc(doused));
    }
}

// Apply an action mask row (bit g % 32 of word g / 32 = water on cell g of the
// context) to the env's planes, all threads; adds the doused cells to *count
// when count is not null.
__device__ void res_action_mask(const uint32_t* __restrict__ mrow, int64_t off, int H, int W, int WW,
                                uint32_t* Bp, uint32_t* D, int tid, int nth, int* count = nullptr) {
    const int words = H * WW;
    const WordDiv wd(WW);
    for (int i = tid; i < words; i += nth) {
        const int y = wd.div(i), w = i - y * WW;
        uint32_t* bp = &Bp[(y + 1) * WW + w];
        if (*bp == 0u) continue;
        const uint32_t m = mask_run(mrow, off + (int64_t)y * W + (w << 5), min(32, W - (w << 5)));
        const uint32_t doused = *bp & m;
        *bp &= ~m;
        D[i] |= doused;
        if (count != nullptr && doused != 0u) atomicAdd(count, __popc(doused));
    }
}

// Chunk activity after a (re)load: flag[c] = chunk c of B holds a burning
// cell; the other buffer's flags get `other` (0 after zeroing, 1 when it may
// hold stale words).  Adds popc(D) to *burnt.  All threads; caller syncs.
__device__ void res_init_flags(const uint32_t* Bp, const uint32_t* D, int WW, int words, int nchunks,
                               uint8_t* fl_cur, uint8_t* fl_other, uint8_t other, int* burnt, int tid, int nth) {
    int nd = 0;
    for (int c = tid; c < nchunks; c += nth) {
        uint32_t any = 0u;
        const int i1 = min(words, (c + 1) << 5);
        for (int i = c << 5; i < i1; ++i) {
            any |= Bp[WW + i];
            nd += __popc(D[i]);
        }
        fl_cur[c] = any != 0u;
        fl_other[c] = other;
    }
    atomicAdd(burnt, nd);
}


// One env stepped a.k times by the NT threads of the CTA, its planes and
// queues in the shared region Rg (its ResEnvShared first), wsc = the per-warp
// scratch of the calling warp.
template <int NT, bool FUSED>
__device__ __forceinline__ void res_env(const ResArgs& a, const RateConsts& sK, const int e, uint32_t* Rg,
                                        uint32_t* wsc) {
    const int tid = threadIdx.x;
    ResEnvShared& T = *reinterpret_cast<ResEnvShared*>(Rg);
    const int H = a.H[e], W = a.W[e];
    const int WW = (W + 31) >> 5;
    const WordDiv wd(WW);
    const int pw = (H + 2) * WW;
    const int words = H * WW;
    const int nchunks = (words + 31) >> 5;
    const int lane = tid & 31, warp = tid >> 5;
    constexpr int nw = NT / 32;
    uint32_t* B0 = Rg + kEnvScalarWords;
    uint32_t* B1 = B0 + pw;
    uint32_t* C = B1 + pw;
    uint32_t* D = C + words;
    uint32_t* list = wsc;                                   // per-warp scratch
    uint32_t* ignw = list + kListCap;
    uint32_t* outw = ignw + 32;
    uint32_t* plist = outw + 32;
    // chunk activity flags of the two burning buffers
    uint8_t* flag0 = reinterpret_cast<uint8_t*>(D + words);
    uint8_t* flag1 = flag0 + nchunks;
    // chunks dealt this step and the block-wide queue of work items
    int* clist = reinterpret_cast<int*>(flag0 + 2 * ((nchunks + 3) & ~3));
    uint32_t* Q = reinterpret_cast<uint32_t*>(clist + nchunks);
    const int reach = (WW + 1 + 31) >> 5;                 // chunks a word's neighbours span
    const int64_t off = a.off[e];
    uint8_t* Fe = a.F + off;
    const bool vec = ((W & 31) == 0) && ((off & 15) == 0);

    // zero both burning planes (the padding rows must read as 0), then load
    for (int i = tid; i < 2 * pw; i += NT) B0[i] = 0u;
    if (tid < 9) T.cnt[tid / 3][tid % 3] = 0;
    if (tid < 3) {
        T.qn[tid] = 0;
        T.ncl[tid] = 0;
    }
    if (tid == 0) T.burnt = 0;
    __syncthreads();
    res_load(Fe, H, W, WW, vec, B0, C, D, tid, NT);
    __syncthreads();
    if (a.drops != nullptr && a.k > 0) {
        res_action(H, W, WW, B0, D, a.drops[(int64_t)e * 2], a.drops[(int64_t)e * 2 + 1], a.R, tid, NT);
        __syncthreads();
    } else if (a.mask != nullptr && a.k > 0) {
        res_action_mask(a.mask, off, H, W, WW, B0, D, tid, NT);
        __syncthreads();
    }
    res_init_flags(B0, D, WW, words, nchunks, flag0, flag1, 0, &T.burnt, tid, NT);
    __syncthreads();
    if (tid == 0) {
        T.burnt_now = T.burnt;
        T.last_burnt = 0;
        T.last_nb = 0;
    }
    uint8_t* fl_c = flag0;
    uint8_t* fl_n = flag1;

    int32_t t = a.t[e];
    int32_t ep = a.episode[e];
    uint32_t* Bc = B0;
    uint32_t* Bn = B1;
    int hist_done = 0;          // history rows written
    const bool rec = a.history != nullptr;
    for (int s = 0; s < a.k; ++s) {
        const uint32_t tt = (uint32_t)t;
        const uint32_t ep4 = 4u * (uint32_t)ep;
        if (rec && s > 0) {
            // record the state after step s - 1, then apply step s's drop
            // (when recording it is not folded into the previous write-back)
            res_record(a, s - 1, off, H, W, WW, vec, Bc, C, D, tid, NT);
            hist_done = s;
            if (tid == 0) T.dous = 0;
            __syncthreads();
            if (a.drops != nullptr) {
                res_action(H, W, WW, Bc, D, a.drops[((int64_t)s * a.N + e) * 2],
                           a.drops[((int64_t)s * a.N + e) * 2 + 1], a.R, tid, NT, &T.dous);
                __syncthreads();
                if (tid == 0) T.burnt_now += T.dous;
            } else if (a.mask != nullptr) {
                res_action_mask(a.mask + (int64_t)s * a.mask_words, off, H, W, WW, Bc, D, tid, NT, &T.dous);
                __syncthreads();
                if (tid == 0) T.burnt_now += T.dous;
            }
        }
        // the next step's drop is applied while the new planes are written:
        // its centre is copied to shared memory while phases A and B run
        const bool next_act = s + 1 < a.k && !rec;
        if (tid == 0) {
            T.cnt[(s + 1) % 3][0] = 0;
            T.cnt[(s + 1) % 3][1] = 0;
            T.cnt[(s + 1) % 3][2] = 0;
            T.qn[(s + 1) % 3] = 0;
            T.ncl[(s + 1) % 3] = 0;
            if (a.drops != nullptr && next_act) {
                const int32_t* dsrc = a.drops + ((int64_t)(s + 1) * a.N + e) * 2;
                jwf_cp_async4(reinterpret_cast<float*>(&T.drop[0]), reinterpret_cast<const float*>(dsrc));
                jwf_cp_async4(reinterpret_cast<float*>(&T.drop[1]), reinterpret_cast<const float*>(dsrc + 1));
            } else {
                T.drop[0] = -1;
                T.drop[1] = -1;
            }
        }
        int my_b = 0, my_o = 0, my_x = 0;
        // phase A: the chunks that can change are dealt to the warps,
        // which clear their words of the write buffer and queue their
        // work items.  A chunk with no burning cell within reach, whose
        // write buffer holds no burning word, cannot change: it is
        // skipped.  Every warp finds the needed chunks of a group of 32
        // with one ballot (lane = chunk); the k-th needed chunk goes to
        // warp k mod (warps), which also lists it for the write-back.
        int n_need = 0;                       // needed chunks before this group
        for (int g0 = 0; g0 < nchunks; g0 += 32) {
            const int cl = g0 + lane;
            bool nd = false;
            if (cl < nchunks) {
                nd = fl_n[cl] != 0;
                for (int cc = max(cl - reach, 0); cc <= min(cl + reach, nchunks - 1); ++cc) nd |= fl_c[cc] != 0;
            }
            const uint32_t need_m = __ballot_sync(0xffffffffu, nd);
            const int rk = n_need + __popc(need_m & ((1u << lane) - 1u));
            const bool take = nd && (rk & (nw - 1)) == warp;
            if (take) clist[rk] = cl;
            n_need += __popc(need_m);
            for (uint32_t mine = __ballot_sync(0xffffffffu, take); mine != 0u;) {
            const int c = g0 + __ffs(mine) - 1;
            mine &= mine - 1u;
            const int base = c << 5;
            const int i = base + lane;
            uint32_t burn = 0, cand = 0;
            uint32_t sd[8];
            if (i < words) {
                const int yw = wd.div(i), w = i - yw * WW;
                const uint32_t* bp = &Bc[WW + i];             // row y + 1 of the padded plane
                const bool hl = w > 0, hr = w + 1 < WW;
                const uint32_t bc = bp[0], bl = hl ? bp[-1] : 0u, br = hr ? bp[1] : 0u;
                const uint32_t uc = bp[-WW], ul = hl ? bp[-WW - 1] : 0u, ur = hr ? bp[-WW + 1] : 0u;
                const uint32_t dc = bp[WW], dl = hl ? bp[WW - 1] : 0u, dr = hr ? bp[WW + 1] : 0u;
                // source of direction d for target (y, x) sits at (y - DR[d], x - DX[d])
                sd[0] = (bc << 1) | (bl >> 31);   // E : (y,   x-1)
                sd[1] = (dc << 1) | (dl >> 31);   // NE: (y+1, x-1)
                sd[2] = dc;                       // N : (y+1, x)
                sd[3] = (dc >> 1) | (dr << 31);   // NW: (y+1, x+1)
                sd[4] = (bc >> 1) | (br << 31);   // W : (y,   x+1)
                sd[5] = (uc >> 1) | (ur << 31);   // SW: (y-1, x+1)
                sd[6] = uc;                       // S : (y-1, x)
                sd[7] = (uc << 1) | (ul >> 31);   // SE: (y-1, x-1)
                const uint32_t any = sd[0] | sd[1] | sd[2] | sd[3] | sd[4] | sd[5] | sd[6] | sd[7];
                cand = C[i] & any;
                if (FUSED && cand != 0u) {
                    // the landcover and elevation of the candidates and of their
                    // sources' rows, wanted by phase B
                    const int64_t g = off + (int64_t)yw * W + (w << 5);
                    asm volatile("prefetch.global.L1 [%0];" ::"l"(a.dem + g));
                    asm volatile("prefetch.global.L1 [%0];" ::"l"(a.cls + g));
                    if (yw > 0) {
                        asm volatile("prefetch.global.L1 [%0];" ::"l"(a.dem + g - W));
                        asm volatile("prefetch.global.L1 [%0];" ::"l"(a.cls + g - W));
                    }
                    if (yw + 1 < H) {
                        asm volatile("prefetch.global.L1 [%0];" ::"l"(a.dem + g + W));
                        asm volatile("prefetch.global.L1 [%0];" ::"l"(a.cls + g + W));
                    }
                }
                burn = bc;
                Bn[WW + i] = 0u;                  // collects this step's ignitions
            } else {
#pragma unroll
                for (int d = 0; d < 8; ++d) sd[d] = 0u;
            }
            __syncwarp();
            uint32_t np = 0;
#pragma unroll
            for (int d = 0; d < 8; ++d) np += __popc(sd[d] & cand);
            if (a.counts != nullptr) {
                // work of the chunk: pairs compared, candidate Philox blocks, burning-cell draws
                const uint32_t cp = __reduce_add_sync(0xffffffffu, np);
                const uint32_t cb = __reduce_add_sync(0xffffffffu, __popc(cand & (sd[0] | sd[1] | sd[2] | sd[3])) +
                                                                       __popc(cand & (sd[4] | sd[5] | sd[6] | sd[7])));
                const uint32_t cd = __reduce_add_sync(0xffffffffu, __popc(burn));
                if (lane == 0) {
                    atomicAdd(&a.counts[0], (unsigned long long)cp);
                    atomicAdd(&a.counts[1], (unsigned long long)cb);
                    atomicAdd(&a.counts[2], (unsigned long long)cd);
                    atomicAdd(&a.counts[3], 32ull);
                }
            }
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
            if (lane == 0) old = atomicAdd(&T.qn[s % 3], total);
            old = __shfl_sync(0xffffffffu, old, 0);
            const int pos = old + total <= kResQCap ? old : -1;
            if (pos < 0) {
                for (int j = old + lane; j < min(kResQCap, old + total); j += 32) Q[j] = kResVoid;
            } else {
                uint32_t* q = Q + pos + (incl - n_items);
                const uint32_t hi = (uint32_t)i << 18;
                for (uint32_t m = burn; m != 0u; m &= m - 1u) *q++ = hi | ((uint32_t)(__ffs(m) - 1) << 13);
                if (FUSED) {
#pragma unroll
                    for (int d = 0; d < 8; ++d)
                        for (uint32_t m = sd[d] & cand; m != 0u; m &= m - 1u)
                            *q++ = hi | ((uint32_t)(__ffs(m) - 1) << 13) | (1u << 12) | (uint32_t)d;
                } else {
                    for (uint32_t m = cand; m != 0u; m &= m - 1u) {
                        const int j = __ffs(m) - 1;
                        uint32_t dm = 0;
#pragma unroll
                        for (int d = 0; d < 8; ++d) dm |= ((sd[d] >> j) & 1u) << d;
                        *q++ = hi | ((uint32_t)j << 13) | (1u << 12) | dm;
                    }
                }
                continue;
            }
            // the queue is full: this warp evaluates the chunk itself
            // (ignitions into the cleared write-buffer words, burn-outs
            // into the burned plane)
            uint32_t* ignw_c = Bn + WW + base;
            uint32_t* outw_c = D + base;
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
                    const int yy = wd.div(ii);
                    const int xx = ((ii - yy * WW) << 5) + j;
                    const uint32_t cell = (uint32_t)(yy * W + xx);
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
                        fused_pairs(a, sK, list, plist, ignw_c, it0, n_pass, base, e, off, W, WW, 0, 0, tt,
                                    ep4, lane);
                }
                __syncwarp();
            }
            }
        }
        if (tid == 0) T.ncl[s % 3] = n_need;
        __syncthreads();
        // phase B: every thread of the CTA evaluates queued items
        {
            const int qn = min(T.qn[s % 3], kResQCap);
            for (int q = tid; q < qn; q += NT) {
                const uint32_t it = Q[q];
                if (it == kResVoid) continue;
                const int ii = (int)(it >> 18), j = (int)(it >> 13) & 31;
                const int yy = wd.div(ii);
                const int xx = ((ii - yy * WW) << 5) + j;
                const bool pair = (it & (1u << 12)) != 0u;
                if (FUSED) {
                    const bool below = item_below(a, sK, e, off, W, yy, xx, pair, (int)(it & 7u), tt, ep4);
                    if (pair && below) atomicOr(&Bn[WW + ii], 1u << j);
                    if (!pair && !below) atomicOr(&D[ii], 1u << j);
                } else {
                    const uint32_t cell = (uint32_t)(yy * W + xx);
                    if (!pair) {
                        const uint4 u = jwf_philox(make_uint4(cell, tt, (uint32_t)e, ep4 + 2u), a.key0, a.key1);
                        if (!(jwf_u24(u.x) < a.p_continue)) atomicOr(&D[ii], 1u << j);
                    } else if (ignites(a, e, off, cell, it & 0xFFu, tt, ep4)) {
                        atomicOr(&Bn[WW + ii], 1u << j);
                    }
                }
            }
        }
        if (tid == 0) asm volatile("cp.async.wait_all;\n" ::: "memory");    // the next step's drop
        __syncthreads();
        // phase C: the dealt chunks are written back, round-robin over the warps
        {
            const int ncl = T.ncl[s % 3];
            const int cxn = T.drop[0], cyn = T.drop[1];
            const uint32_t* mrow =
                (a.mask != nullptr && next_act) ? a.mask + (int64_t)(s + 1) * a.mask_words : nullptr;
            for (int k = warp; k < ncl; k += nw) {
                const int c = clist[k];
                const int i = (c << 5) + lane;
                uint32_t nb = 0u;
                if (i < words) {
                    const int y = wd.div(i), w = i - y * WW;
                    const uint32_t burn = Bc[WW + i];
                    const uint32_t ig = Bn[WW + i];
                    const uint32_t ou = D[i] & burn;          // burning cells that burned out
                    nb = (burn & ~ou) | ig;
                    my_b += __popc(nb);
                    my_o += __popc(ou);
                    const uint32_t m = mrow != nullptr
                                           ? mask_run(mrow, off + (int64_t)y * W + (w << 5), min(32, W - (w << 5)))
                                           : drop_bits(y, w, W, cxn, cyn, a.R);
                    const uint32_t doused = nb & m;
                    my_x += __popc(doused);
                    nb &= ~m;
                    Bn[WW + i] = nb;
                    D[i] |= doused;
                    C[i] &= ~ig;
                }
                const uint32_t any_nb = __ballot_sync(0xffffffffu, nb != 0u);
                if (lane == 0) fl_n[c] = any_nb != 0u;
            }
        }
        my_b = __reduce_add_sync(0xffffffffu, my_b);
        my_o = __reduce_add_sync(0xffffffffu, my_o);
        my_x = __reduce_add_sync(0xffffffffu, my_x);
        if (lane == 0) {
            atomicAdd(&T.cnt[s % 3][0], my_b);
            atomicAdd(&T.cnt[s % 3][1], my_o);
            atomicAdd(&T.cnt[s % 3][2], my_x);
        }
        __syncthreads();
        const int32_t nb = T.cnt[s % 3][0];
        uint32_t* tmp = Bc;
        Bc = Bn;
        Bn = tmp;
        uint8_t* ftmp = fl_c;
        fl_c = fl_n;
        fl_n = ftmp;
        t += 1;
        const bool done = (nb == 0) || (a.t_max > 0 && t >= a.t_max);
        if (tid == 0) {
            const int32_t nd = T.burnt_now + T.cnt[s % 3][1];     // burned after the step
            T.burnt_now = nd + T.cnt[s % 3][2];                  // and after the next drop
            T.last_burnt = nd;
            T.last_nb = nb;
            const int64_t o = (int64_t)s * a.N + e;
            if (a.out_burning) a.out_burning[o] = nb;
            if (a.out_burnt) a.out_burnt[o] = nd;
            if (a.out_done) a.out_done[o] = done ? 1 : 0;
        }
        if (done && a.auto_reset) {
            // restart from the initial state with a fresh random stream
            t = 0;
            ep += 1;
            for (int i2 = tid; i2 < pw; i2 += NT) Bc[i2] = 0u;
            if (tid == 0) T.burnt = 0;
            __syncthreads();
            res_load(a.F0 + off, H, W, WW, vec, Bc, C, D, tid, NT);
            __syncthreads();
            if (T.drop[0] >= 0) {
                res_action(H, W, WW, Bc, D, T.drop[0], T.drop[1], a.R, tid, NT);
                __syncthreads();
            } else if (a.mask != nullptr && next_act) {
                res_action_mask(a.mask + (int64_t)(s + 1) * a.mask_words, off, H, W, WW, Bc, D, tid, NT);
                __syncthreads();
            }
            // the other buffer may hold stale burning words: mark it active
            res_init_flags(Bc, D, WW, words, nchunks, fl_c, fl_n, 1, &T.burnt, tid, NT);
            __syncthreads();
            if (tid == 0) T.burnt_now = T.burnt;
            continue;
        }
        if (nb == 0) {
            // fire out: nothing can change any more; fill the remaining steps
            __syncthreads();
            const int32_t last_burnt = T.last_burnt;
            for (int s2 = s + 1 + tid; s2 < a.k; s2 += NT) {
                const int64_t o = (int64_t)s2 * a.N + e;
                if (a.out_burning) a.out_burning[o] = 0;
                if (a.out_burnt) a.out_burnt[o] = last_burnt;
                if (a.out_done) a.out_done[o] = 1;
            }
            t += a.k - (s + 1);
            break;
        }
    }
    __syncthreads();
    res_store(Fe, H, W, WW, vec, Bc, C, D, tid, NT);
    if (a.history != nullptr) {
        // the last step's state, and the unchanged state of the steps after the fire went out
        for (int j = hist_done; j < a.k; ++j) res_record(a, j, off, H, W, WW, vec, Bc, C, D, tid, NT);
    }
    if (tid == 0) {
        a.t[e] = t;
        a.episode[e] = ep;
        if (a.last_burning != nullptr) a.last_burning[e] = T.last_nb;
    }
    __syncthreads();
}

// Persistent CTAs pull envs from the work queue and step each one with all
// NT threads.  At most 64 registers a thread: 1024 threads fit an SM.
template <int NT, bool FUSED>
__global__ void __launch_bounds__(NT, 1024 / NT)
k_step_resident(const ResArgs a, const RateConsts Kc) {
    extern __shared__ uint32_t sm[];
    // the rate constants live in shared memory only in the fused variant
    __shared__ typename std::conditional<FUSED, RateConsts, int>::type sK_store;
    const RateConsts& sK = *reinterpret_cast<const RateConsts*>(&sK_store);
    if (FUSED) {
        for (int i = threadIdx.x; i < (int)(sizeof(RateConsts) / 4); i += NT)
            reinterpret_cast<float*>(&sK_store)[i] = reinterpret_cast<const float*>(&Kc)[i];
    }
    // per-warp scratch first, then the env's region (its ResEnvShared first)
    uint32_t* wsc = sm + (threadIdx.x >> 5) * kWarpScratch;
    uint32_t* Rg = sm + (NT / 32) * kWarpScratch;
    ResEnvShared& T = *reinterpret_cast<ResEnvShared*>(Rg);
    for (;;) {
        if (threadIdx.x == 0) {
            const uint32_t slot = atomicAdd(&a.queue[0], 1u);
            T.env = slot < (uint32_t)a.nq ? a.order[slot] : -1;
        }
        __syncthreads();
        const int e = T.env;
        __syncthreads();
        if (e < 0) break;
        res_env<NT, FUSED>(a, sK, e, Rg, wsc);
    }
    __syncthreads();
    // the last CTA to leave resets the queue for the next launch
    if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t fin = atomicAdd(&a.queue[1], 1u);
        if (fin == gridDim.x - 1) {
            a.queue[0] = 0u;
            a.queue[1] = 0u;
            __threadfence();
        }
    }
}

constexpr int kMaxDev = 64;

// Per-instantiation launch facts, cached per device so that a launch after
// the first one makes no attribute or occupancy query.
template <int NT, bool FUSED>
cudaError_t launch_t(const jwf_ctx* c, const ResArgs& a, const RateConsts& K, size_t smem, cudaStream_t s,
                     int32_t nq) {
    constexpr int kSlots = 8;
    static size_t set_smem[kMaxDev] = {};
    static size_t occ_smem[kMaxDev][kSlots] = {};
    static int occ_blocks[kMaxDev][kSlots] = {};
    const int dev = c->device;
    if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
    cudaError_t err;
    if (smem > set_smem[dev]) {
        err = cudaFuncSetAttribute(k_step_resident<NT, FUSED>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
        set_smem[dev] = smem;
    }
    int slot = -1;
    for (int i = 0; i < kSlots; ++i)
        if (occ_blocks[dev][i] > 0 && occ_smem[dev][i] == smem) slot = i;
    if (slot < 0) {
        int per_sm = 0;
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_resident<NT, FUSED>, NT, smem);
        if (err != cudaSuccess) return err;
        slot = 0;
        for (int i = 0; i < kSlots; ++i)
            if (occ_blocks[dev][i] == 0) { slot = i; break; }
        occ_blocks[dev][slot] = per_sm;
        occ_smem[dev][slot] = smem;
    }
    if (occ_blocks[dev][slot] < 1) return cudaErrorInvalidConfiguration;
    int64_t grid = (int64_t)occ_blocks[dev][slot] * c->num_sms;
    if (grid > nq) grid = nq;
    k_step_resident<NT, FUSED><<<(unsigned)grid, NT, smem, s>>>(a, K);
    return cudaGetLastError();
}

template <bool FUSED>
cudaError_t launch_v(const jwf_ctx* c, int threads, const ResArgs& a, const RateConsts& K, size_t smem,
                     cudaStream_t s, int32_t nq) {
    switch (threads) {
        case 32: return launch_t<32, FUSED>(c, a, K, smem, s, nq);
        case 64: return launch_t<64, FUSED>(c, a, K, smem, s, nq);
        case 128: return launch_t<128, FUSED>(c, a, K, smem, s, nq);
        case 256: return launch_t<256, FUSED>(c, a, K, smem, s, nq);
        case 512: return launch_t<512, FUSED>(c, a, K, smem, s, nq);
        case 1024: return launch_t<1024, FUSED>(c, a, K, smem, s, nq);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

void jwf_rate_consts(const jwf_ctx* c, RateConsts* K);


size_t jwf_resident_smem(int32_t H, int32_t W, int threads) {
    // queued work items address words with 14 bits
    if ((int64_t)H * ((W + 31) / 32) >= (int64_t)1 << 14) return (size_t)1 << 40;
    return (size_t)(res_region_words(H, W) + (threads / 32) * kWarpScratch) * sizeof(uint32_t);
}

int jwf_resident_threads(int32_t H, int32_t W) {
    const int64_t words = (int64_t)H * ((W + 31) / 32);
    if (words <= 64) return 32;
    if (words <= 256) return 64;
    if (words <= 2048) return 128;
    return 256;
}

// Reorder each size class's envs by the burning count after the first part
// of a split launch, largest first (envs whose fire is out go last): one CTA
// per class, a counting sort over min(count, kSortKeys - 1).  Only the speed
// depends on the order.
constexpr int kSortKeys = 1024;

__global__ void __launch_bounds__(1024) k_reorder(const int32_t* __restrict__ order_in, int32_t* __restrict__ order_out,
                                                  const int32_t* __restrict__ last_burning, int4 starts, int4 counts) {
    __shared__ int32_t hist[kSortKeys];
    const int g = blockIdx.x;
    const int start = g == 0 ? starts.x : g == 1 ? starts.y : g == 2 ? starts.z : starts.w;
    const int n = g == 0 ? counts.x : g == 1 ? counts.y : g == 2 ? counts.z : counts.w;
    for (int i = threadIdx.x; i < kSortKeys; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    // bin (kSortKeys - 1 - key): larger counts first
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int key = min(last_burning[order_in[start + i]], kSortKeys - 1);
        atomicAdd(&hist[kSortKeys - 1 - key], 1);
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        // exclusive scan of the bins by one warp (32 bins a lane)
        const int lane = threadIdx.x;
        int sum = 0;
        for (int j = 0; j < kSortKeys / 32; ++j) sum += hist[lane * (kSortKeys / 32) + j];
        int incl = sum;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        int run = incl - sum;
        for (int j = 0; j < kSortKeys / 32; ++j) {
            const int b = lane * (kSortKeys / 32) + j;
            const int h = hist[b];
            hist[b] = run;
            run += h;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int e = order_in[start + i];
        const int key = min(last_burning[e], kSortKeys - 1);
        order_out[start + atomicAdd(&hist[kSortKeys - 1 - key], 1)] = e;
    }
}

cudaError_t launch_resident_part(jwf_ctx* c, int32_t k, const int32_t* drops, const uint32_t* masks,
                                 int32_t* burning, int32_t* burnt, uint8_t* done, const int32_t* order,
                                 int32_t* last_burning, cudaStream_t s);

cudaError_t jwf_launch_step_resident(jwf_ctx* c, int32_t k, const int32_t* drops, const uint32_t* masks,
                                     int32_t* burning, int32_t* burnt, uint8_t* done, cudaStream_t s) {
    const int32_t k1 = c->reorder_steps;
    const int ng = (int)c->groups.size();
    // (one size class only: with several, the classes run on forked streams
    // and the reorder would join them between the two parts)
    if (k1 <= 0 || k < 2 * k1 || c->hist != nullptr || c->d_lastb == nullptr || ng != 1)
        return launch_resident_part(c, k, drops, masks, burning, burnt, done, c->d_order, nullptr, s);
    // two launches: k1 steps in the creation order, then the rest with the
    // envs whose fires are largest after k1 steps first (the longest fires
    // set the end of the launch, so they should not start last)
    cudaError_t err = launch_resident_part(c, k1, drops, masks, burning, burnt, done, c->d_order, c->d_lastb, s);
    if (err != cudaSuccess) return err;
    int st[4] = {0, 0, 0, 0}, cn[4] = {0, 0, 0, 0};
    for (int g = 0; g < ng; ++g) {
        st[g] = c->groups[g].start;
        cn[g] = c->groups[g].count;
    }
    k_reorder<<<ng, 1024, 0, s>>>(c->d_order, c->d_order_dyn, c->d_lastb, make_int4(st[0], st[1], st[2], st[3]),
                                  make_int4(cn[0], cn[1], cn[2], cn[3]));
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    const int64_t o = (int64_t)k1 * c->N;
    const uint32_t* m2 = masks ? masks + (int64_t)k1 * jwf_mask_row_words(c->cells) : nullptr;
    return launch_resident_part(c, k - k1, drops ? drops + 2 * o : nullptr, m2, burning ? burning + o : nullptr,
                                burnt ? burnt + o : nullptr, done ? done + o : nullptr, c->d_order_dyn, nullptr, s);
}

cudaError_t launch_resident_part(jwf_ctx* c, int32_t k, const int32_t* drops, const uint32_t* masks,
                                 int32_t* burning, int32_t* burnt, uint8_t* done, const int32_t* order,
                                 int32_t* last_burning, cudaStream_t s) {
    const bool fused = c->kernel == JWF_KERNEL_FUSED;
    ResArgs a;
    a.last_burning = last_burning;
    a.H = c->d_H;
    a.W = c->d_W;
    a.off = c->d_off;
    a.N = c->N;
    a.F = c->d_state[c->cur];
    a.F0 = c->d_F0;
    a.q = c->d_q;
    a.cls = c->t_cls;
    a.dem = c->t_dem;
    a.wexp = c->wser_n > 0 ? c->d_wser : c->d_wexp;
    a.wser_n = c->wser_n;
    a.drops = drops;
    a.mask = masks;
    a.mask_words = jwf_mask_row_words(c->cells);
    a.t = c->d_t;
    a.episode = c->d_episode;
    a.out_burning = burning;
    a.out_burnt = burnt;
    a.out_done = done;
    a.counts = c->d_pairs;
    a.k = k;
    a.t_max = c->t_max;
    a.R = c->drop_radius;
    a.auto_reset = (c->flags & JWF_AUTO_RESET) ? 1 : 0;
    a.key0 = (uint32_t)(c->seed & 0xffffffffu);
    a.key1 = (uint32_t)(c->seed >> 32);
    a.p_continue = c->P.p_continue;
    a.history = c->hist;
    a.cells = c->cells;
    a.hist_packed = c->hist_packed ? 1 : 0;
    a.hist_stride = c->hist_packed ? jwf_packed_bytes(c->cells) : c->cells;
    a.packed_aligned = c->packed_aligned ? 1 : 0;
    if (c->hist != nullptr && c->hist_packed && !c->packed_aligned) {
        // rows are assembled by OR from words that share bytes
        const cudaError_t e0 = cudaMemsetAsync(c->hist, 0, (size_t)k * (size_t)a.hist_stride, s);
        if (e0 != cudaSuccess) return e0;
    }
    RateConsts K;
    if (fused)
        jwf_rate_consts(c, &K);
    else
        K = RateConsts{};
    // one persistent launch per size class; classes run side by side on
    // forked streams when there is more than one
    const int ng = (int)c->groups.size();
    cudaError_t err = cudaSuccess;
    if (ng > 1) {
        err = cudaEventRecord(c->ev_fork, s);
        if (err != cudaSuccess) return err;
    }
    for (int g = 0; g < ng; ++g) {
        const JwfGroup& G = c->groups[g];
        int threads = c->threads_per_env > 0 ? c->threads_per_env
                                             : (G.threads > 0 ? G.threads : jwf_resident_threads(G.maxH, G.maxW));
        if (threads != 32 && threads != 64 && threads != 128 && threads != 512 && threads != 1024) threads = 256;
        const size_t smem = jwf_resident_smem(G.maxH, G.maxW, threads);
        cudaStream_t gs = s;
        if (ng > 1) {
            gs = c->side[g];
            err = cudaStreamWaitEvent(gs, c->ev_fork, 0);
            if (err != cudaSuccess) return err;
        }
        a.order = order + G.start;
        a.nq = G.count;
        a.queue = c->d_queue + 2 * g;
        err = fused ? launch_v<true>(c, threads, a, K, smem, gs, G.count)
                    : launch_v<false>(c, threads, a, K, smem, gs, G.count);
        if (err != cudaSuccess) return err;
        if (ng > 1) {
            err = cudaEventRecord(c->ev_join[g], gs);
            if (err == cudaSuccess) err = cudaStreamWaitEvent(s, c->ev_join[g], 0);
            if (err != cudaSuccess) return err;
        }
    }
    return cudaSuccess;
}
