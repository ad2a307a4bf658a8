// k_step.cu -- discrete (stochastic) update of Section 3 with the tanker
// action of Section 4.
//
// Two step kernels give identical results (the random numbers are
// counter-based, so neither cell order nor skipped work changes them):
//
//  * k_step_plain: one launch per step, one thread per cell, state in global
//    memory (ping-pong buffers).  The reference GPU path.
//
//  * k_step_resident (k_resident.cu): whole envs in shared memory as bit
//    planes, k steps per launch.
#include "jwf_internal.cuh"

namespace {

__global__ void k_load(const int64_t cells, const uint8_t* __restrict__ F0, uint8_t* __restrict__ Fc,
                       uint8_t* __restrict__ F0c, int32_t* __restrict__ t, int32_t* __restrict__ ep,
                       int32_t N) {
    // 16 cells per thread when the three buffers are 16-byte aligned
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool vec = ((reinterpret_cast<uintptr_t>(F0) | reinterpret_cast<uintptr_t>(Fc) |
                       reinterpret_cast<uintptr_t>(F0c)) & 15u) == 0;
    if (vec) {
        const int64_t n16 = cells >> 4;
        if (i < n16) {
            const uint4 v = __ldg(reinterpret_cast<const uint4*>(F0) + i);
            reinterpret_cast<uint4*>(Fc)[i] = v;
            reinterpret_cast<uint4*>(F0c)[i] = v;
        }
        const int64_t tail = (n16 << 4) + i;
        if (i < 16 && tail < cells) {
            Fc[tail] = F0[tail];
            F0c[tail] = F0[tail];
        }
    } else {
        for (int64_t j = i; j < cells; j += (int64_t)gridDim.x * blockDim.x) {
            const uint8_t s = F0[j];
            Fc[j] = s;
            F0c[j] = s;
        }
    }
    if (i < N) {
        t[i] = 0;
        ep[i] = 0;
    }
}

// ---------------------------------------------------------------------------
// 2-bit packed states: cell i in bits 2(i mod 4), 2(i mod 4) + 1 of byte i/4
// ---------------------------------------------------------------------------
// four states in the bytes of v -> their 8 packed bits
__device__ __forceinline__ uint32_t pack4(uint32_t v) {
    uint32_t x = v & 0x03030303u;
    x = (x | (x >> 6)) & 0x000f000fu;
    return (x | (x >> 12)) & 0xffu;
}

// 8 packed bits -> four states in the bytes of the result
__device__ __forceinline__ uint32_t unpack4(uint32_t p) {
    uint32_t x = p & 0xffu;
    x = (x | (x << 12)) & 0x000f000fu;
    return (x | (x << 6)) & 0x03030303u;
}

// n states -> ceil(n / 4) packed bytes (only the low two bits of a state are
// kept); 16 states a thread when F is 16-byte and P 4-byte aligned
__global__ void k_pack(const int64_t n, const uint8_t* __restrict__ F, uint8_t* __restrict__ P) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool vec = ((reinterpret_cast<uintptr_t>(F) & 15u) | (reinterpret_cast<uintptr_t>(P) & 3u)) == 0;
    const int64_t n16 = vec ? (n >> 4) : 0;
    for (int64_t i = i0; i < n16; i += stride) {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(F) + i);
        reinterpret_cast<uint32_t*>(P)[i] = pack4(v.x) | (pack4(v.y) << 8) | (pack4(v.z) << 16) | (pack4(v.w) << 24);
    }
    const int64_t nb = (n + 3) >> 2;
    for (int64_t b = n16 * 4 + i0; b < nb; b += stride) {
        uint32_t x = 0;
        for (int j = 0; j < 4; ++j) {
            const int64_t c = 4 * b + j;
            if (c < n) x |= (uint32_t)(F[c] & 3u) << (2 * j);
        }
        P[b] = (uint8_t)x;
    }
}

// ceil(n / 4) packed bytes -> n states in F (and F2 when not null); with t and
// ep not null also the start of a run (t = episode = 0 for the N envs)
__global__ void k_unpack(const int64_t n, const uint8_t* __restrict__ P, uint8_t* __restrict__ F,
                         uint8_t* __restrict__ F2, int32_t* __restrict__ t, int32_t* __restrict__ ep, int32_t N) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uintptr_t al = (reinterpret_cast<uintptr_t>(F) & 15u) | (reinterpret_cast<uintptr_t>(F2) & 15u) |
                         (reinterpret_cast<uintptr_t>(P) & 3u);
    const int64_t n16 = al == 0 ? (n >> 4) : 0;
    for (int64_t i = i0; i < n16; i += stride) {
        const uint32_t w = __ldg(reinterpret_cast<const uint32_t*>(P) + i);
        const uint4 v = make_uint4(unpack4(w), unpack4(w >> 8), unpack4(w >> 16), unpack4(w >> 24));
        reinterpret_cast<uint4*>(F)[i] = v;
        if (F2 != nullptr) reinterpret_cast<uint4*>(F2)[i] = v;
    }
    for (int64_t c = n16 * 16 + i0; c < n; c += stride) {
        const uint8_t v = (uint8_t)((P[c >> 2] >> (2 * (c & 3))) & 3u);
        F[c] = v;
        if (F2 != nullptr) F2[c] = v;
    }
    if (t != nullptr)
        for (int64_t j = i0; j < N; j += stride) {
            t[j] = 0;
            ep[j] = 0;
        }
}

// uint8 masks [n_rows][cells] (nonzero = water) -> bit rows of
// jwf_mask_row_words(cells) words: one ballot per 32 cells
__global__ void k_pack_masks(int32_t n_rows, int64_t cells, int64_t words, const uint8_t* __restrict__ m,
                             uint32_t* __restrict__ bits) {
    const int64_t total = (int64_t)n_rows * words * 32;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // whole warps walk the cells 32 at a time (the loop bound is a multiple of 32)
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i - (threadIdx.x & 31) < total; i += stride) {
        const int64_t r = i / (words * 32), g = i - r * words * 32;
        const bool on = g < cells && m[r * cells + g] != 0;
        const uint32_t b = __ballot_sync(0xffffffffu, on);
        if ((threadIdx.x & 31) == 0) bits[r * words + (g >> 5)] = b;
    }
}

unsigned pack_blocks(int64_t work) {
    int64_t b = (work + 255) / 256;
    if (b < 1) b = 1;
    return (unsigned)(b > 152 * 16 ? 152 * 16 : b);
}

__global__ void k_reset(const int2* __restrict__ tiles, const int32_t* __restrict__ Hs,
                        const int32_t* __restrict__ Ws, const int64_t* __restrict__ offs,
                        const uint8_t* __restrict__ env_mask, const uint8_t* __restrict__ F0,
                        uint8_t* __restrict__ F) {
    const int2 tile = tiles[blockIdx.x];
    const int e = tile.x;
    if (env_mask != nullptr && env_mask[e] == 0) return;
    const int local = tile.y + (int)threadIdx.x;
    if (local >= Hs[e] * Ws[e]) return;
    const int64_t v = offs[e] + local;
    F[v] = F0[v];
}

__global__ void k_reset_counters(const uint8_t* __restrict__ env_mask, int32_t* __restrict__ t,
                                 int32_t* __restrict__ ep, int32_t N) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N) return;
    if (env_mask != nullptr && env_mask[e] == 0) return;
    t[e] = 0;
    ep[e] += 1;
}

__global__ void k_action(const int64_t cells, const uint8_t* __restrict__ mask, uint8_t* __restrict__ F) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cells && mask[i] != 0 && F[i] == 2) F[i] = 3;
}

// ---------------------------------------------------------------------------
// Plain step: one launch per step, state in global memory (reads F_t, writes
// F_{t+1}), the q table read for the cells that can ignite.  A thread steps a
// segment of up to 16 cells of one row: the three rows around it are read as
// 16-byte vectors where they are aligned (byte by byte otherwise) and the
// burning sources after the step's drop become bit masks, so that a cell's
// eight sources are bit tests.  Counts: one shared-memory reduction and one
// atomic per block and counter into cnt[0][e] (burning), cnt[1][e] (burned);
// k_finalize turns them into the per-step outputs.
// ---------------------------------------------------------------------------
constexpr int kSeg = JWF_PLAIN_SEG;

// 4 states (one word) -> 4-bit mask of the bytes equal to `pattern`
__device__ __forceinline__ uint32_t eq4(uint32_t w, uint32_t pattern) {
    const uint32_t m = __vcmpeq4(w, pattern);
    return (((m & 0x01010101u) * 0x01020408u) >> 24) & 0xFu;
}
// 4-bit mask -> 4 bytes of 0 / 1
__device__ __forceinline__ uint32_t spread4(uint32_t n) { return (n * 0x00204081u) & 0x01010101u; }

// Row y over columns x0 - 1 .. x0 + kSeg: masks (bit k + 1 = column x0 + k,
// bit 0 = x0 - 1, bit n + 1 = x0 + n) of the cells in state 1, 2 and 3;
// rows and columns outside the grid are 0
struct RowBits {
    uint32_t c, b, d;
};
__device__ __forceinline__ RowBits row_bits(const uint8_t* __restrict__ Fe, int y, int x0, int n, int H, int W,
                                            bool vec) {
    RowBits r = {0u, 0u, 0u};
    if (y < 0 || y >= H) return r;
    const uint8_t* row = Fe + (int64_t)y * W;
    if (vec) {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(row + x0));
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            r.c |= eq4(w[j], 0x01010101u) << (4 * j + 1);
            r.b |= eq4(w[j], 0x02020202u) << (4 * j + 1);
            r.d |= eq4(w[j], 0x03030303u) << (4 * j + 1);
        }
    } else {
        for (int k = 0; k < n; ++k) {
            const uint32_t st = row[x0 + k];
            r.c |= (uint32_t)(st == 1) << (k + 1);
            r.b |= (uint32_t)(st == 2) << (k + 1);
            r.d |= (uint32_t)(st == 3) << (k + 1);
        }
    }
    if (x0 > 0 && row[x0 - 1] == 2) r.b |= 1u;
    if (x0 + n < W && row[x0 + n] == 2) r.b |= 1u << (n + 1);
    return r;
}

// bits [lo, hi] of an 18-bit row mask (columns cx - R .. cx + R) doused by the
// step's drop, or 0 when the row or the drop is out of reach
__device__ __forceinline__ uint32_t drop_mask(int y, int x0, int cx, int cy, int R) {
    if (cx < 0 || cy < 0 || abs(y - cy) > R) return 0u;
    const int lo = max(cx - R - x0 + 1, 0), hi = min(cx + R - x0 + 1, kSeg + 1);
    if (lo > hi) return 0u;
    return ((hi - lo == 31) ? 0xffffffffu : ((1u << (hi - lo + 1)) - 1u)) << lo;
}

// the action mask row's bits for columns x0 - 1 .. x0 + n of row y (the bit
// layout of row_bits), columns and rows outside the grid 0
__device__ __forceinline__ uint32_t mask_bits(const uint32_t* __restrict__ mrow, int64_t off, int y, int x0, int n,
                                              int H, int W) {
    if (y < 0 || y >= H) return 0u;
    const int c0 = max(x0 - 1, 0), c1 = min(x0 + n, W - 1);
    return mask_run(mrow, off + (int64_t)y * W + c0, c1 - c0 + 1) << (c0 - x0 + 1);
}

__global__ void __launch_bounds__(JWF_TILE)
k_step_plain(const int2* __restrict__ tiles, const int32_t* __restrict__ Hs,
             const int32_t* __restrict__ Ws, const int64_t* __restrict__ offs, int32_t N,
             const uint8_t* __restrict__ Fin, uint8_t* __restrict__ Fout,
             const float* __restrict__ q, const int32_t* __restrict__ drops, const uint32_t* __restrict__ mrow,
             const int32_t* __restrict__ tcur, const int32_t* __restrict__ episode,
             uint32_t key0, uint32_t key1, float p_continue, int R, int32_t* __restrict__ cnt) {
    __shared__ int32_t s_n[2];
    const int2 tile = tiles[blockIdx.x];
    const int e = tile.x;
    const int W = Ws[e], H = Hs[e];
    const int segs = (W + kSeg - 1) / kSeg;
    if (threadIdx.x < 2) s_n[threadIdx.x] = 0;
    __syncthreads();
    int cx = -1, cy = -1;
    if (drops != nullptr) {
        cx = drops[2 * e];
        cy = drops[2 * e + 1];
    }
    const int64_t off = offs[e];
    const uint32_t t = (uint32_t)tcur[e];
    const uint32_t ep4 = 4u * (uint32_t)episode[e];
    const uint8_t* Fe = Fin + off;
    int nb = 0, nd = 0;
    // the block's JWF_PLAIN_SEGS_PER_THREAD x JWF_TILE consecutive segments of the env
#pragma unroll 1
    for (int i = 0; i < JWF_PLAIN_SEGS_PER_THREAD; ++i) {
        const int u = tile.y + i * JWF_TILE + (int)threadIdx.x;      // segment of the env
        if (u >= H * segs) break;
        const int y = u / segs;
        const int x0 = (u - y * segs) * kSeg;
        const int n = min(kSeg, W - x0);
        const uint32_t nmask = n == 32 ? 0xffffffffu : ((1u << n) - 1u);
        // rows start on 16-byte boundaries and the segment is whole
        const bool vec = n == kSeg && ((off | (int64_t)W) & 15) == 0;
        const RowBits ru = row_bits(Fe, y - 1, x0, n, H, W, vec);
        const RowBits rc = row_bits(Fe, y, x0, n, H, W, vec);
        const RowBits rd = row_bits(Fe, y + 1, x0, n, H, W, vec);
        // burning sources after the step's action (burning under water -> burned)
        const uint32_t mdu = mrow ? mask_bits(mrow, off, y - 1, x0, n, H, W) : drop_mask(y - 1, x0, cx, cy, R);
        const uint32_t mdr = mrow ? mask_bits(mrow, off, y, x0, n, H, W) : drop_mask(y, x0, cx, cy, R);
        const uint32_t mdd = mrow ? mask_bits(mrow, off, y + 1, x0, n, H, W) : drop_mask(y + 1, x0, cx, cy, R);
        const uint32_t mu = ru.b & ~mdu;
        const uint32_t mc = rc.b & ~mdr;
        const uint32_t md = rd.b & ~mdd;
        // the segment's own cells (bit k = column x0 + k)
        const uint32_t own_c = (rc.c >> 1) & nmask;
        const uint32_t own_b = (mc >> 1) & nmask;                           // burning after the drop
        const uint32_t own_d = ((rc.d | (rc.b & mdr)) >> 1) & nmask;        // burned, or doused now
        // can-burn cells with a burning source: bit k of a row mask is column
        // x0 + k - 1, so cell k's sources sit at bits k, k + 1, k + 2
        const uint32_t any = mc | (mc >> 2) | md | (md >> 1) | (md >> 2) | mu | (mu >> 1) | (mu >> 2);
        const uint32_t cand = own_c & any;
        uint32_t ign = 0u, outb = 0u;
        const uint32_t row0 = (uint32_t)(y * W + x0);
        for (uint32_t m = cand; m != 0u; m &= m - 1u) {
            const int k = __ffs(m) - 1;
            // sources of directions 0..7: (y, x-1), (y+1, x-1), (y+1, x), (y+1, x+1), (y, x+1),
            // (y-1, x+1), (y-1, x), (y-1, x-1)
            const uint32_t dm = ((mc >> k) & 1u) | (((md >> k) & 1u) << 1) | (((md >> (k + 1)) & 1u) << 2) |
                                (((md >> (k + 2)) & 1u) << 3) | (((mc >> (k + 2)) & 1u) << 4) |
                                (((mu >> (k + 2)) & 1u) << 5) | (((mu >> (k + 1)) & 1u) << 6) |
                                (((mu >> k) & 1u) << 7);
            const uint32_t local = row0 + (uint32_t)k;
            const float4* q4 = reinterpret_cast<const float4*>(q + (off + local) * 8);
            bool hit = false;
            if (dm & 0x0Fu) {
                const uint4 r = jwf_philox(make_uint4(local, t, (uint32_t)e, ep4 + 0u), key0, key1);
                const float4 qa = __ldg(q4);
                hit |= ((dm & 1u) && jwf_u24(r.x) < qa.x) || ((dm & 2u) && jwf_u24(r.y) < qa.y) ||
                       ((dm & 4u) && jwf_u24(r.z) < qa.z) || ((dm & 8u) && jwf_u24(r.w) < qa.w);
            }
            if (!hit && (dm & 0xF0u)) {
                const uint4 r = jwf_philox(make_uint4(local, t, (uint32_t)e, ep4 + 1u), key0, key1);
                const float4 qb = __ldg(q4 + 1);
                hit |= ((dm & 16u) && jwf_u24(r.x) < qb.x) || ((dm & 32u) && jwf_u24(r.y) < qb.y) ||
                       ((dm & 64u) && jwf_u24(r.z) < qb.z) || ((dm & 128u) && jwf_u24(r.w) < qb.w);
            }
            if (hit) ign |= 1u << k;
        }
        for (uint32_t m = own_b; m != 0u; m &= m - 1u) {
            const int k = __ffs(m) - 1;
            const uint4 r = jwf_philox(make_uint4(row0 + (uint32_t)k, t, (uint32_t)e, ep4 + 2u), key0, key1);
            if (!(jwf_u24(r.x) < p_continue)) outb |= 1u << k;
        }
        // the next states: 1 can burn, 2 burning, 3 burned (0 stays 0)
        const uint32_t s1 = own_c & ~ign;
        const uint32_t s2 = (own_b & ~outb) | ign;
        const uint32_t s3 = own_d | outb;
        nb += __popc(s2);
        nd += __popc(s3);
        uint32_t w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int sh = 4 * j;
            w[j] = spread4((s1 >> sh) & 0xFu) + 2u * spread4((s2 >> sh) & 0xFu) + 3u * spread4((s3 >> sh) & 0xFu);
        }
        uint8_t* dst = Fout + off + (int64_t)y * W + x0;
        if (vec) {
            *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
        } else {
            for (int k = 0; k < n; ++k) dst[k] = (uint8_t)(w[k >> 2] >> (8 * (k & 3)));
        }
    }
    // a block never straddles two envs: one atomic per counter
    nb = __reduce_add_sync(0xffffffffu, nb);
    nd = __reduce_add_sync(0xffffffffu, nd);
    if ((threadIdx.x & 31) == 0) {
        if (nb) atomicAdd(&s_n[0], nb);
        if (nd) atomicAdd(&s_n[1], nd);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_n[0]) atomicAdd(&cnt[e], s_n[0]);
        if (s_n[1]) atomicAdd(&cnt[N + e], s_n[1]);
    }
}

// per-env bookkeeping after a plain step: outputs, t += 1, done, reset flag
__global__ void k_finalize(int32_t N, int32_t* __restrict__ cnt, int32_t* __restrict__ t,
                           int32_t* __restrict__ ep, int32_t t_max, int auto_reset,
                           int32_t* __restrict__ burning, int32_t* __restrict__ burnt,
                           uint8_t* __restrict__ done, uint8_t* __restrict__ flag) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N) return;
    const int32_t nb = cnt[e], nd = cnt[N + e];
    cnt[e] = 0;
    cnt[N + e] = 0;
    const int32_t tn = t[e] + 1;
    const bool is_done = (nb == 0) || (t_max > 0 && tn >= t_max);
    if (burning) burning[e] = nb;
    if (burnt) burnt[e] = nd;
    if (done) done[e] = is_done ? 1 : 0;
    if (is_done && auto_reset) {
        t[e] = 0;
        ep[e] += 1;
        flag[e] = 1;
    } else {
        t[e] = tn;
        flag[e] = 0;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t jwf_launch_load(jwf_ctx* c, const uint8_t* F0, cudaStream_t s) {
    const int64_t n16 = (c->cells + 15) / 16;
    const int64_t n = n16 > c->N ? n16 : c->N;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    c->cur = 0;
    k_load<<<blocks, 256, 0, s>>>(c->cells, F0, c->d_state[0], c->d_F0, c->d_t, c->d_episode, c->N);
    return cudaGetLastError();
}

cudaError_t jwf_launch_pack(int64_t n, const uint8_t* states, uint8_t* packed, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_pack<<<pack_blocks((n + 15) / 16), 256, 0, s>>>(n, states, packed);
    return cudaGetLastError();
}

cudaError_t jwf_launch_unpack(int64_t n, const uint8_t* packed, uint8_t* states, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_unpack<<<pack_blocks((n + 15) / 16), 256, 0, s>>>(n, packed, states, nullptr, nullptr, nullptr, 0);
    return cudaGetLastError();
}

cudaError_t jwf_launch_load_packed(jwf_ctx* c, const uint8_t* P0, cudaStream_t s) {
    const int64_t w = (c->cells + 15) / 16;
    c->cur = 0;
    k_unpack<<<pack_blocks(w > c->N ? w : c->N), 256, 0, s>>>(c->cells, P0, c->d_state[0], c->d_F0, c->d_t,
                                                              c->d_episode, c->N);
    return cudaGetLastError();
}

cudaError_t jwf_record_row(jwf_ctx* c, int64_t row, cudaStream_t s) {
    if (c->hist_packed)
        return jwf_launch_pack(c->cells, c->d_state[c->cur], c->hist + row * jwf_packed_bytes(c->cells), s);
    return cudaMemcpyAsync(c->hist + row * c->cells, c->d_state[c->cur], (size_t)c->cells,
                           cudaMemcpyDeviceToDevice, s);
}

cudaError_t jwf_launch_reset(jwf_ctx* c, const uint8_t* env_mask, cudaStream_t s) {
    k_reset<<<(unsigned)c->n_tiles, JWF_TILE, 0, s>>>(c->d_tiles, c->d_H, c->d_W, c->d_off, env_mask,
                                                       c->d_F0, c->d_state[c->cur]);
    k_reset_counters<<<(c->N + 255) / 256, 256, 0, s>>>(env_mask, c->d_t, c->d_episode, c->N);
    return cudaGetLastError();
}

cudaError_t jwf_launch_action(jwf_ctx* c, const uint8_t* mask, cudaStream_t s) {
    k_action<<<(unsigned)((c->cells + 255) / 256), 256, 0, s>>>(c->cells, mask, c->d_state[c->cur]);
    return cudaGetLastError();
}

cudaError_t jwf_launch_step_plain(jwf_ctx* c, int32_t k, const int32_t* drops, const uint32_t* masks,
                                  int32_t* burning, int32_t* burnt, uint8_t* done, cudaStream_t s) {
    const int64_t mw = jwf_mask_row_words(c->cells);
    const uint32_t key0 = (uint32_t)(c->seed & 0xffffffffu), key1 = (uint32_t)(c->seed >> 32);
    const int auto_reset = (c->flags & JWF_AUTO_RESET) ? 1 : 0;
    for (int32_t st = 0; st < k; ++st) {
        const uint8_t* Fin = c->d_state[c->cur];
        uint8_t* Fout = c->d_state[c->cur ^ 1];
        k_step_plain<<<(unsigned)c->n_ptiles, JWF_TILE, 0, s>>>(
            c->d_ptiles, c->d_H, c->d_W, c->d_off, c->N, Fin, Fout, c->d_q,
            drops ? drops + (int64_t)st * c->N * 2 : nullptr, masks ? masks + (int64_t)st * mw : nullptr, c->d_t,
            c->d_episode, key0, key1,
            c->P.p_continue, c->drop_radius, c->d_cnt);
        const int64_t o = (int64_t)st * c->N;
        k_finalize<<<(c->N + 255) / 256, 256, 0, s>>>(
            c->N, c->d_cnt, c->d_t, c->d_episode, c->t_max, auto_reset, burning ? burning + o : nullptr,
            burnt ? burnt + o : nullptr, done ? done + o : nullptr, c->d_flag);
        c->cur ^= 1;
        if (auto_reset) {
            k_reset<<<(unsigned)c->n_tiles, JWF_TILE, 0, s>>>(c->d_tiles, c->d_H, c->d_W, c->d_off,
                                                               c->d_flag, c->d_F0, c->d_state[c->cur]);
        }
        cudaError_t err = cudaGetLastError();
        if (err == cudaSuccess && c->hist != nullptr) err = jwf_record_row(c, st, s);
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

// Discrete states -> relaxed planes: p_un = [no fuel or can burn], p_burn =
// [burning] (p_bd = [burned] is implicit), e.g. for a straight-through
// backward along a sampled trajectory.
__global__ void k_state_planes(int64_t n, const uint8_t* __restrict__ st, float* __restrict__ pun,
                               float* __restrict__ pburn) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint8_t v = st[i];
        pun[i] = v <= 1 ? 1.0f : 0.0f;
        pburn[i] = v == 2 ? 1.0f : 0.0f;
    }
}

cudaError_t jwf_launch_state_planes(int64_t n, const uint8_t* states, float* pun, float* pburn, cudaStream_t s) {
    int64_t blocks = (n + 255) / 256;
    if (blocks > 65536) blocks = 65536;
    k_state_planes<<<(unsigned)blocks, 256, 0, s>>>(n, states, pun, pburn);
    return cudaGetLastError();
}

cudaError_t jwf_launch_pack_masks(int32_t n_rows, int64_t cells, const uint8_t* masks, uint32_t* bits,
                                  cudaStream_t s) {
    const int64_t words = jwf_mask_row_words(cells);
    if (n_rows <= 0 || words == 0) return cudaSuccess;
    k_pack_masks<<<pack_blocks((int64_t)n_rows * words * 32), 256, 0, s>>>(n_rows, cells, words, masks, bits);
    return cudaGetLastError();
}
