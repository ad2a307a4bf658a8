// k_step.cu -- discrete (stochastic) update of Section 3 with the tanker
// action of Section 4.
//
// Two step kernels give identical results (the random numbers are
// counter-based, so neither cell order nor skipped work changes them):
//
//  * k_step_plain: one launch per step, one thread per cell, state in global
//    memory (ping-pong buffers).  The reference GPU path.
//
//  * k_step_resident: persistent CTAs pull whole envs from a work queue
//    (largest first), keep the env in shared memory as bit planes (burning,
//    can-burn, burned; 32 cells per word) and run k steps per launch.
//    A step is word-parallel: each lane owns one 32-cell word, finds the
//    can-burn cells with a burning neighbour and the burning cells with 8
//    shifted ORs, and the warp then shares out the active cells (ballot +
//    prefix sum) so that every lane draws Philox numbers and reads q rows for
//    the same number of cells.  An env whose fire is out stops early (its
//    state can no longer change); with auto-reset it restarts instead.
#include "jwf_internal.cuh"

namespace {

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool in_drop(int y, int x, int cx, int cy, int R) {
    return cx >= 0 && cy >= 0 && abs(y - cy) <= R && abs(x - cx) <= R;
}

// state after the action of this step (burning under the drop -> burned)
__device__ __forceinline__ uint8_t acted(uint8_t s, int y, int x, int cx, int cy, int R) {
    return (s == 2 && in_drop(y, x, cx, cy, R)) ? (uint8_t)3 : s;
}

__global__ void k_load(const int64_t cells, const uint8_t* __restrict__ F0, uint8_t* __restrict__ Fc,
                       uint8_t* __restrict__ F0c, int32_t* __restrict__ t, int32_t* __restrict__ ep,
                       int32_t N) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cells) {
        const uint8_t s = F0[i];
        Fc[i] = s;
        F0c[i] = s;
    }
    if (i < N) {
        t[i] = 0;
        ep[i] = 0;
    }
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
// Plain step: one thread per cell, reads F_t (global), writes F_{t+1}.
// Counts go to cnt[0][e] (burning) and cnt[1][e] (burned) by warp-aggregated
// atomics; k_finalize turns them into the per-step outputs.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(JWF_TILE)
k_step_plain(const int2* __restrict__ tiles, const int32_t* __restrict__ Hs,
             const int32_t* __restrict__ Ws, const int64_t* __restrict__ offs, int32_t N,
             const uint8_t* __restrict__ Fin, uint8_t* __restrict__ Fout,
             const float* __restrict__ q, const int32_t* __restrict__ drops,
             const int32_t* __restrict__ tcur, const int32_t* __restrict__ episode,
             uint32_t key0, uint32_t key1, float p_continue, int R, int32_t* __restrict__ cnt) {
    const int2 tile = tiles[blockIdx.x];
    const int e = tile.x;
    const int W = Ws[e], H = Hs[e];
    const int local = tile.y + (int)threadIdx.x;
    const bool valid = local < H * W;
    int cx = -1, cy = -1;
    if (drops != nullptr) {
        cx = drops[2 * e];
        cy = drops[2 * e + 1];
    }
    uint8_t nxt = 0;
    if (valid) {
        const int64_t off = offs[e];
        const int y = local / W, x = local - (local / W) * W;
        const uint8_t s = acted(Fin[off + local], y, x, cx, cy, R);
        nxt = s;
        const uint32_t t = (uint32_t)tcur[e];
        const uint32_t ep4 = 4u * (uint32_t)episode[e];
        if (s == 1) {
            uint32_t dm = 0;
#pragma unroll
            for (int d = 0; d < 8; ++d) {
                const int uy = y - jwf_dr(d), ux = x - jwf_dx(d);
                if (uy < 0 || uy >= H || ux < 0 || ux >= W) continue;
                const uint8_t su = acted(Fin[off + (int64_t)uy * W + ux], uy, ux, cx, cy, R);
                if (su == 2) dm |= 1u << d;
            }
            if (dm != 0) {
                const float4* q4 = reinterpret_cast<const float4*>(q + (off + local) * 8);
                bool ign = false;
                if (dm & 0x0Fu) {
                    const uint4 u = jwf_philox(make_uint4((uint32_t)local, t, (uint32_t)e, ep4 + 0u), key0, key1);
                    const float4 qa = __ldg(q4);
                    ign |= ((dm & 1u) && jwf_u24(u.x) < qa.x) || ((dm & 2u) && jwf_u24(u.y) < qa.y) ||
                           ((dm & 4u) && jwf_u24(u.z) < qa.z) || ((dm & 8u) && jwf_u24(u.w) < qa.w);
                }
                if (dm & 0xF0u) {
                    const uint4 u = jwf_philox(make_uint4((uint32_t)local, t, (uint32_t)e, ep4 + 1u), key0, key1);
                    const float4 qb = __ldg(q4 + 1);
                    ign |= ((dm & 16u) && jwf_u24(u.x) < qb.x) || ((dm & 32u) && jwf_u24(u.y) < qb.y) ||
                           ((dm & 64u) && jwf_u24(u.z) < qb.z) || ((dm & 128u) && jwf_u24(u.w) < qb.w);
                }
                if (ign) nxt = 2;
            }
        } else if (s == 2) {
            const uint4 u = jwf_philox(make_uint4((uint32_t)local, t, (uint32_t)e, ep4 + 2u), key0, key1);
            nxt = (jwf_u24(u.x) < p_continue) ? (uint8_t)2 : (uint8_t)3;
        }
        Fout[off + local] = nxt;
    }
    // a block never straddles two envs
    const uint32_t b2 = __ballot_sync(0xffffffffu, valid && nxt == 2);
    const uint32_t b3 = __ballot_sync(0xffffffffu, valid && nxt == 3);
    if ((threadIdx.x & 31) == 0) {
        if (b2) atomicAdd(&cnt[e], __popc(b2));
        if (b3) atomicAdd(&cnt[N + e], __popc(b3));
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

// ---------------------------------------------------------------------------
// Resident k-step kernel.
// ---------------------------------------------------------------------------
constexpr int kListCap = 256;   // active cells shared out per warp pass

struct ResArgs {
    const int32_t* H;
    const int32_t* W;
    const int64_t* off;
    const int32_t* order;
    int32_t N;
    uint8_t* F;                 // in/out (in place: one CTA per env)
    const uint8_t* F0;
    const float* q;
    const int32_t* drops;       // [k][N][2] or null
    int32_t* t;
    int32_t* episode;
    int32_t* out_burning;       // [k][N] or null
    int32_t* out_burnt;
    uint8_t* out_done;
    uint32_t* queue;            // [0] cursor, [1] CTAs finished
    unsigned long long* pairs;  // optional: count of q entries compared
    int32_t k;
    int32_t t_max;
    int32_t R;
    int32_t auto_reset;
    uint32_t key0, key1;
    float p_continue;
};

// Shared-memory layout for one env of H rows and WW = ceil(W/32) words:
//   Bp[2][(H+2)*(WW+2)]  burning plane, zero-padded ring, double-buffered
//   C[H*WW], D[H*WW]     can-burn and burned planes (updated in place)
//   per warp: list[kListCap], ign[32], out[32]
__host__ __device__ __forceinline__ int res_plane_words(int H, int W) {
    const int WW = (W + 31) >> 5;
    return 2 * (H + 2) * (WW + 2) + 2 * H * WW;
}

// Load env into planes: each thread handles whole words.
__device__ void res_load(const uint8_t* __restrict__ Fe, int H, int W, int WW, int P,
                         uint32_t* Bp, uint32_t* C, uint32_t* D) {
    const int words = H * WW;
    for (int i = threadIdx.x; i < words; i += blockDim.x) {
        const int y = i / WW, w = i - (i / WW) * WW;
        const int x0 = w << 5;
        const int n = min(32, W - x0);
        const uint8_t* src = Fe + (int64_t)y * W + x0;
        uint32_t b = 0, c = 0, dd = 0;
        for (int j = 0; j < n; ++j) {
            const uint32_t s = src[j];
            b |= (uint32_t)(s == 2) << j;
            c |= (uint32_t)(s == 1) << j;
            dd |= (uint32_t)(s == 3) << j;
        }
        Bp[(y + 1) * P + (w + 1)] = b;
        C[i] = c;
        D[i] = dd;
    }
}

__device__ void res_store(uint8_t* __restrict__ Fe, int H, int W, int WW, int P,
                          const uint32_t* Bp, const uint32_t* C, const uint32_t* D) {
    const int words = H * WW;
    for (int i = threadIdx.x; i < words; i += blockDim.x) {
        const int y = i / WW, w = i - (i / WW) * WW;
        const int x0 = w << 5;
        const int n = min(32, W - x0);
        uint8_t* dst = Fe + (int64_t)y * W + x0;
        const uint32_t b = Bp[(y + 1) * P + (w + 1)], c = C[i], dd = D[i];
        for (int j = 0; j < n; ++j)
            dst[j] = (uint8_t)(((c >> j) & 1u) * 1u + ((b >> j) & 1u) * 2u + ((dd >> j) & 1u) * 3u);
    }
}

// Apply a drop of radius R centred at (cx, cy) to the burning plane: cells
// under it that burn become burned.  Called by one warp.
__device__ void res_action(int H, int W, int WW, int P, uint32_t* Bp, uint32_t* D, int cx, int cy,
                           int R) {
    if (cx < 0 || cy < 0) return;
    const int lane = threadIdx.x & 31;
    const int y0 = max(cy - R, 0), y1 = min(cy + R, H - 1);
    const int x0 = max(cx - R, 0), x1 = min(cx + R, W - 1);
    if (y0 > y1 || x0 > x1) return;
    const int w0 = x0 >> 5, w1 = x1 >> 5;
    const int nw = w1 - w0 + 1;
    const int total = (y1 - y0 + 1) * nw;
    for (int j = lane; j < total; j += 32) {
        const int y = y0 + j / nw, w = w0 + j % nw;
        const int lo = max(x0 - (w << 5), 0), hi = min(x1 - (w << 5), 31);
        const uint32_t m = (hi - lo == 31) ? 0xffffffffu : (((1u << (hi - lo + 1)) - 1u) << lo);
        uint32_t* bp = &Bp[(y + 1) * P + (w + 1)];
        const uint32_t doused = *bp & m;
        *bp &= ~m;
        D[y * WW + w] |= doused;
    }
}

__global__ void __launch_bounds__(256)
k_step_resident(const ResArgs a) {
    extern __shared__ uint32_t sm[];
    __shared__ int32_t s_env;
    __shared__ int32_t s_cnt[3][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;

    for (;;) {
        if (threadIdx.x == 0) {
            const uint32_t slot = atomicAdd(&a.queue[0], 1u);
            s_env = (slot < (uint32_t)a.N) ? a.order[slot] : -1;
        }
        __syncthreads();
        const int e = s_env;
        __syncthreads();
        if (e < 0) break;

        const int H = a.H[e], W = a.W[e];
        const int WW = (W + 31) >> 5, P = WW + 2;
        const int pw = (H + 2) * P;
        uint32_t* B0 = sm;
        uint32_t* B1 = B0 + pw;
        uint32_t* C = B1 + pw;
        uint32_t* D = C + H * WW;
        uint32_t* wl = D + H * WW + warp * (kListCap + 64);   // per-warp scratch
        uint32_t* list = wl;
        uint32_t* ignw = wl + kListCap;
        uint32_t* outw = ignw + 32;
        const int64_t off = a.off[e];
        uint8_t* Fe = a.F + off;
        const int words = H * WW;

        // zero both burning planes (the padding ring must read as 0), then load
        for (int i = threadIdx.x; i < 2 * pw; i += blockDim.x) B0[i] = 0u;
        __syncthreads();
        res_load(Fe, H, W, WW, P, B0, C, D);
        if (threadIdx.x < 6) s_cnt[threadIdx.x / 2][threadIdx.x & 1] = 0;
        // per-warp ign/out words start cleared
        ignw[lane] = 0u;
        outw[lane] = 0u;
        __syncthreads();

        int32_t t = a.t[e];
        int32_t ep = a.episode[e];
        uint32_t* Bc = B0;
        uint32_t* Bn = B1;
        int s = 0;
        int32_t last_burnt = 0;
        for (; s < a.k; ++s) {
            // 1. action of this step on the current planes (one warp), then sync
            if (a.drops != nullptr && warp == 0) {
                const int cx = a.drops[((int64_t)s * a.N + e) * 2];
                const int cy = a.drops[((int64_t)s * a.N + e) * 2 + 1];
                res_action(H, W, WW, P, Bc, D, cx, cy, a.R);
            }
            if (threadIdx.x == 0) {
                s_cnt[(s + 1) % 3][0] = 0;
                s_cnt[(s + 1) % 3][1] = 0;
            }
            __syncthreads();

            // 2. spread and burn-out, chunk of 32 words per warp pass
            const uint32_t tt = (uint32_t)t;
            const uint32_t ep4 = 4u * (uint32_t)ep;
            int my_b = 0, my_d = 0;
            uint32_t my_pairs = 0;
            for (int base = warp * 32; base < words; base += nwarps * 32) {
                const int i = base + lane;
                uint32_t burn = 0, cand = 0;
                uint32_t sd[8];
                int y = 0, w = 0;
                if (i < words) {
                    y = i / WW;
                    w = i - y * WW;
                    const uint32_t* bp = &Bc[(y + 1) * P + (w + 1)];
                    const uint32_t bc = bp[0], bl = bp[-1], br = bp[1];
                    const uint32_t uc = bp[-P], ul = bp[-P - 1], ur = bp[-P + 1];
                    const uint32_t dc = bp[P], dl = bp[P - 1], dr = bp[P + 1];
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
                    burn = bc;
                } else {
#pragma unroll
                    for (int d = 0; d < 8; ++d) sd[d] = 0u;
                }
                const uint32_t act = cand | burn;
                const uint32_t bal = __ballot_sync(0xffffffffu, act != 0u);
                if (bal != 0u) {
                    // share out the active cells of these 32 words across the warp
                    const int n_act = __popc(act);
                    int incl = n_act;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int v = __shfl_up_sync(0xffffffffu, incl, o);
                        if (lane >= o) incl += v;
                    }
                    const int total = __shfl_sync(0xffffffffu, incl, 31);
                    const int excl = incl - n_act;
                    for (int pass = 0; pass < total; pass += kListCap) {
                        // write this lane's items that fall into [pass, pass + cap)
                        uint32_t rem = act;
                        int idx = excl;
                        while (rem != 0u) {
                            const int j = __ffs(rem) - 1;
                            rem &= rem - 1u;
                            if (idx >= pass && idx < pass + kListCap) {
                                uint32_t item = ((uint32_t)lane << 5) | (uint32_t)j;  // 10 bits
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
                        const int n_pass = min(kListCap, total - pass);
                        for (int it = lane; it < n_pass; it += 32) {
                            const uint32_t item = list[it];
                            const int ol = (int)(item >> 5) & 31;     // owner lane
                            const int j = (int)item & 31;
                            const int ii = base + ol;                 // word index
                            const int yy = ii / WW;
                            const int xx = ((ii - yy * WW) << 5) + j;
                            const uint32_t cell = (uint32_t)(yy * W + xx);
                            if (item & (1u << 18)) {
                                const uint32_t dm = (item >> 10) & 0xFFu;
                                my_pairs += __popc(dm);
                                const float4* q4 = reinterpret_cast<const float4*>(a.q + (off + cell) * 8);
                                bool ign = false;
                                if (dm & 0x0Fu) {
                                    const uint4 u = jwf_philox(make_uint4(cell, tt, (uint32_t)e, ep4), a.key0, a.key1);
                                    const float4 qa = __ldg(q4);
                                    ign |= ((dm & 1u) && jwf_u24(u.x) < qa.x) || ((dm & 2u) && jwf_u24(u.y) < qa.y) ||
                                           ((dm & 4u) && jwf_u24(u.z) < qa.z) || ((dm & 8u) && jwf_u24(u.w) < qa.w);
                                }
                                if (dm & 0xF0u) {
                                    const uint4 u = jwf_philox(make_uint4(cell, tt, (uint32_t)e, ep4 + 1u), a.key0, a.key1);
                                    const float4 qb = __ldg(q4 + 1);
                                    ign |= ((dm & 16u) && jwf_u24(u.x) < qb.x) || ((dm & 32u) && jwf_u24(u.y) < qb.y) ||
                                           ((dm & 64u) && jwf_u24(u.z) < qb.z) || ((dm & 128u) && jwf_u24(u.w) < qb.w);
                                }
                                if (ign) atomicOr(&ignw[ol], 1u << j);
                            } else {
                                const uint4 u = jwf_philox(make_uint4(cell, tt, (uint32_t)e, ep4 + 2u), a.key0, a.key1);
                                if (!(jwf_u24(u.x) < a.p_continue)) atomicOr(&outw[ol], 1u << j);
                            }
                        }
                        __syncwarp();
                    }
                }
                if (i < words) {
                    const uint32_t ig = ignw[lane], ou = outw[lane];
                    const uint32_t nb = (burn & ~ou) | ig;
                    Bn[(y + 1) * P + (w + 1)] = nb;
                    const uint32_t nd = D[i] | ou;
                    D[i] = nd;
                    C[i] &= ~ig;
                    ignw[lane] = 0u;
                    outw[lane] = 0u;
                    my_b += __popc(nb);
                    my_d += __popc(nd);
                }
                __syncwarp();
            }
            // 3. counts
            if (a.pairs != nullptr) {
                my_pairs = __reduce_add_sync(0xffffffffu, my_pairs);
                if (lane == 0 && my_pairs) atomicAdd(a.pairs, (unsigned long long)my_pairs);
            }
            my_b = __reduce_add_sync(0xffffffffu, my_b);
            my_d = __reduce_add_sync(0xffffffffu, my_d);
            if (lane == 0) {
                atomicAdd(&s_cnt[s % 3][0], my_b);
                atomicAdd(&s_cnt[s % 3][1], my_d);
            }
            __syncthreads();
            const int32_t nb = s_cnt[s % 3][0];
            const int32_t nd = s_cnt[s % 3][1];
            uint32_t* tmp = Bc;
            Bc = Bn;
            Bn = tmp;
            t += 1;
            const bool done = (nb == 0) || (a.t_max > 0 && t >= a.t_max);
            if (threadIdx.x == 0) {
                const int64_t o = (int64_t)s * a.N + e;
                if (a.out_burning) a.out_burning[o] = nb;
                if (a.out_burnt) a.out_burnt[o] = nd;
                if (a.out_done) a.out_done[o] = done ? 1 : 0;
            }
            last_burnt = nd;
            if (done && a.auto_reset) {
                // restart from the initial state with a fresh random stream
                t = 0;
                ep += 1;
                for (int i2 = threadIdx.x; i2 < pw; i2 += blockDim.x) Bc[i2] = 0u;
                __syncthreads();
                res_load(a.F0 + off, H, W, WW, P, Bc, C, D);
                __syncthreads();
                continue;
            }
            if (nb == 0) {
                // fire out: nothing can change any more; fill the remaining steps
                for (int s2 = s + 1 + (int)threadIdx.x; s2 < a.k; s2 += blockDim.x) {
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
        res_store(Fe, H, W, WW, P, Bc, C, D);
        if (threadIdx.x == 0) {
            a.t[e] = t;
            a.episode[e] = ep;
        }
        __syncthreads();
    }
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

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t jwf_launch_load(jwf_ctx* c, const uint8_t* F0, cudaStream_t s) {
    const int64_t n = c->cells > c->N ? c->cells : c->N;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    c->cur = 0;
    k_load<<<blocks, 256, 0, s>>>(c->cells, F0, c->d_state[0], c->d_F0, c->d_t, c->d_episode, c->N);
    return cudaGetLastError();
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

cudaError_t jwf_launch_step_plain(jwf_ctx* c, int32_t k, const int32_t* drops, int32_t* burning,
                                  int32_t* burnt, uint8_t* done, cudaStream_t s) {
    const uint32_t key0 = (uint32_t)(c->seed & 0xffffffffu), key1 = (uint32_t)(c->seed >> 32);
    const int auto_reset = (c->flags & JWF_AUTO_RESET) ? 1 : 0;
    for (int32_t st = 0; st < k; ++st) {
        const uint8_t* Fin = c->d_state[c->cur];
        uint8_t* Fout = c->d_state[c->cur ^ 1];
        k_step_plain<<<(unsigned)c->n_tiles, JWF_TILE, 0, s>>>(
            c->d_tiles, c->d_H, c->d_W, c->d_off, c->N, Fin, Fout, c->d_q,
            drops ? drops + (int64_t)st * c->N * 2 : nullptr, c->d_t, c->d_episode, key0, key1,
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
        const cudaError_t err = cudaGetLastError();
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

size_t jwf_resident_smem(int32_t H, int32_t W, int threads) {
    const int nwarps = threads / 32;
    return (size_t)(res_plane_words(H, W) + nwarps * (kListCap + 64)) * sizeof(uint32_t);
}

int jwf_resident_threads(int32_t H, int32_t W) {
    const int64_t words = (int64_t)H * ((W + 31) / 32);
    if (words <= 64) return 64;
    if (words <= 256) return 128;
    return 256;
}

cudaError_t jwf_launch_step_resident(jwf_ctx* c, int32_t k, const int32_t* drops,
                                     int32_t* burning, int32_t* burnt, uint8_t* done,
                                     cudaStream_t s) {
    const int threads = c->threads_per_env > 0 ? c->threads_per_env
                                               : jwf_resident_threads(c->maxH, c->maxW);
    const size_t smem = jwf_resident_smem(c->maxH, c->maxW, threads);
    cudaError_t err = cudaFuncSetAttribute(k_step_resident, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_resident, threads, smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int64_t grid = (int64_t)per_sm * c->num_sms;
    if (grid > c->N) grid = c->N;
    ResArgs a;
    a.H = c->d_H;
    a.W = c->d_W;
    a.off = c->d_off;
    a.order = c->d_order;
    a.N = c->N;
    a.F = c->d_state[c->cur];
    a.F0 = c->d_F0;
    a.q = c->d_q;
    a.drops = drops;
    a.t = c->d_t;
    a.episode = c->d_episode;
    a.out_burning = burning;
    a.out_burnt = burnt;
    a.out_done = done;
    a.queue = c->d_queue;
    a.pairs = c->d_pairs;
    a.k = k;
    a.t_max = c->t_max;
    a.R = c->drop_radius;
    a.auto_reset = (c->flags & JWF_AUTO_RESET) ? 1 : 0;
    a.key0 = (uint32_t)(c->seed & 0xffffffffu);
    a.key1 = (uint32_t)(c->seed >> 32);
    a.p_continue = c->P.p_continue;
    k_step_resident<<<(unsigned)grid, threads, smem, s>>>(a);
    return cudaGetLastError();
}
