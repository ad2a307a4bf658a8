// k_agent.cu -- the air-tanker agent environment of Section 4: an agent moves
// over the grid and controls a valve that drops a limited amount of water; it
// sees an egocentric window of the fire state; each step costs a penalty per
// burning cell and putting the fire out earns +10; episodes restart with a
// random agent position and, optionally, a random ignition.
//
// One agent step = k_agent_act (move, valve, water -> this step's drop
// centre) + one discrete step (jwf_step, which applies the drop first) +
// k_agent_post (reward, agent restart for envs the step restarted,
// observation).  The paper gives the ingredients but not their details; the
// readings (action set, drop footprint, window, restart draws) are:
//   action a in [0, 10): move = a % 5 (0 stay, 1 north = row - 1, 2 east =
//     column + 1, 3 south, 4 west; clamped to the grid), valve open = a >= 5;
//     out-of-range actions count as 0;
//   an open valve with water left drops water on the drop footprint centred
//     on the agent's new cell and uses one unit;
//   observation = the k x k states centred on the agent (255 outside);
//   restart: Philox4x32-10 with the step's key and counter (0, 0, env,
//     4 * episode + 3) gives x = floor(u(w0) W), y = floor(u(w1) H) and, for
//     a random ignition, the first can-burn cell at or after cell
//     floor(u(w2) H W) in row-major order (wrapping) starts burning.
#include <type_traits>

#include "jwf_internal.cuh"
#include "rate_model.cuh"
#include "step_common.cuh"

void jwf_rate_consts(const jwf_ctx* c, RateConsts* K);

namespace {

__global__ void k_agent_act(int32_t N, const int32_t* __restrict__ Hs, const int32_t* __restrict__ Ws,
                            const int32_t* __restrict__ actions, int32_t* __restrict__ agent,
                            int32_t* __restrict__ drops) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N) return;
    int a = actions[e];
    if (a < 0 || a >= 10) a = 0;
    const int H = Hs[e], W = Ws[e];
    int x = agent[e * 3], y = agent[e * 3 + 1], water = agent[e * 3 + 2];
    const int move = a % 5;
    if (move == 1) y -= 1;
    if (move == 2) x += 1;
    if (move == 3) y += 1;
    if (move == 4) x -= 1;
    x = min(max(x, 0), W - 1);
    y = min(max(y, 0), H - 1);
    int cx = -1, cy = -1;
    if (a >= 5 && water > 0) {
        cx = x;
        cy = y;
        water -= 1;
    }
    agent[e * 3] = x;
    agent[e * 3 + 1] = y;
    agent[e * 3 + 2] = water;
    drops[e * 2] = cx;
    drops[e * 2 + 1] = cy;
}

// One warp per env.  mode 0: after a step (reward; restart the agent of envs
// the step restarted); mode 1: restart every env's agent (episode start).
__global__ void k_agent_post(int32_t N, const int32_t* __restrict__ Hs, const int32_t* __restrict__ Ws,
                             const int64_t* __restrict__ offs, uint8_t* __restrict__ F,
                             const int32_t* __restrict__ episode, const int32_t* __restrict__ burning,
                             const uint8_t* __restrict__ done, int auto_reset, int mode, int32_t* __restrict__ agent,
                             int32_t water0, int random_fire, uint32_t key0, uint32_t key1, float burn_penalty,
                             float* __restrict__ reward, int32_t obs_k, uint8_t* __restrict__ obs) {
    const int e = blockIdx.x;
    if (e >= N) return;
    const int lane = threadIdx.x;
    const int H = Hs[e], W = Ws[e];
    const int64_t off = offs[e];
    uint8_t* Fe = F + off;
    bool restart = mode == 1;
    if (mode == 0) {
        const int32_t nb = burning[e];
        if (lane == 0 && reward != nullptr) reward[e] = -burn_penalty * (float)nb + (nb == 0 ? 10.0f : 0.0f);
        restart = auto_reset && done[e] != 0;
    }
    if (restart) {
        const uint4 w = jwf_philox(make_uint4(0u, 0u, (uint32_t)e, 4u * (uint32_t)episode[e] + 3u), key0, key1);
        if (lane == 0) {
            agent[e * 3] = min((int)(jwf_u24(w.x) * (float)W), W - 1);
            agent[e * 3 + 1] = min((int)(jwf_u24(w.y) * (float)H), H - 1);
            agent[e * 3 + 2] = water0;
        }
        if (random_fire) {
            const int n = H * W;
            const int start = min((int)(jwf_u24(w.z) * (float)n), n - 1);
            // first can-burn cell at or after start, row-major, wrapping
            for (int base = 0; base < n; base += 32) {
                const int k = base + lane;
                const int c = k < n ? (start + k) % n : 0;
                const bool hit = k < n && Fe[c] == 1;
                const uint32_t m = __ballot_sync(0xffffffffu, hit);
                if (m != 0u) {
                    if (lane == __ffs(m) - 1) Fe[c] = 2;
                    break;
                }
            }
        }
        __syncwarp();
    }
    if (obs != nullptr) {
        const int x = agent[e * 3], y = agent[e * 3 + 1];
        const int r = obs_k / 2;
        for (int i = lane; i < obs_k * obs_k; i += 32) {
            const int yy = y - r + i / obs_k, xx = x - r + i % obs_k;
            obs[(int64_t)e * obs_k * obs_k + i] = (yy >= 0 && yy < H && xx >= 0 && xx < W) ? Fe[yy * W + xx] : 255;
        }
    }
}


// Fused agent step for grids of at most 32 x 32 cells: one warp per env, one
// row per lane as three bit words (can burn, burning, burned), the source
// masks of the eight directions from the row and its neighbours (shuffles),
// work items shared out across the warp, then reward, restart and
// observation -- one launch per agent step, the same results as
// k_agent_act + the discrete step + k_agent_post.
struct AgentArgs {
    const int32_t* H;
    const int32_t* W;
    const int64_t* off;
    int32_t N;
    uint8_t* F;
    const uint8_t* F0;
    const float* q;             // table variant
    const uint8_t* cls;         // fused variant
    const float* dem;
    const float2* wexp;
    int32_t wser_n;
    int32_t* t;
    int32_t* episode;
    const int32_t* actions;
    int32_t* agent;
    float* reward;
    uint8_t* done;
    uint8_t* obs;
    int32_t obs_k;
    int32_t t_max, R, auto_reset, water0, random_fire;
    uint32_t key0, key1;
    float p_continue, burn_penalty;
};

constexpr int kAgentWarps = 8;
constexpr int kAgentList = 256;

__device__ __forceinline__ uint32_t bits_between(int lo, int hi) {   // bits lo..hi (0 <= lo <= hi <= 31)
    return (hi - lo == 31) ? 0xffffffffu : (((1u << (hi - lo + 1)) - 1u) << lo);
}

// Rows of env state (lane = row) from uint8 cells: the warp copies the grid
// to its shared buffer with coalesced loads, then each lane packs its row.
__device__ __forceinline__ void agent_load_row(const uint8_t* Fe, int H, int W, int lane, uint8_t* buf,
                                               uint32_t& B, uint32_t& C, uint32_t& D) {
    const int n = H * W;
    if ((reinterpret_cast<uintptr_t>(Fe) & 3u) == 0 && (n & 3) == 0) {
        for (int i = lane; i < n / 4; i += 32)
            reinterpret_cast<uint32_t*>(buf)[i] = reinterpret_cast<const uint32_t*>(Fe)[i];
    } else {
        for (int i = lane; i < n; i += 32) buf[i] = Fe[i];
    }
    __syncwarp();
    B = C = D = 0u;
    if (lane < H) {
        const uint8_t* row = buf + lane * W;
        for (int x = 0; x < W; ++x) {
            const uint32_t v = row[x];
            C |= (uint32_t)(v == 1) << x;
            B |= (uint32_t)(v == 2) << x;
            D |= (uint32_t)(v == 3) << x;
        }
    }
    __syncwarp();
}

// (at most 48 registers a thread: five CTAs, 40 warps, per SM; four at 64
// registers ran 3% slower, six at 40 spilled more and ran slower still)
template <bool FUSED>
__global__ void __launch_bounds__(kAgentWarps * 32, 5)
k_agent_warp(const AgentArgs a, const RateConsts Kc) {
    __shared__ typename std::conditional<FUSED, RateConsts, int>::type sK_store;
    __shared__ __align__(16) uint8_t s_cells[kAgentWarps][32 * 32];
    __shared__ uint32_t s_list[kAgentWarps][kAgentList];
    __shared__ uint32_t s_ig[kAgentWarps][32], s_ou[kAgentWarps][32];
    const RateConsts& sK = *reinterpret_cast<const RateConsts*>(&sK_store);
    if (FUSED) {
        for (int i = threadIdx.x; i < (int)(sizeof(RateConsts) / 4); i += blockDim.x)
            reinterpret_cast<float*>(&sK_store)[i] = reinterpret_cast<const float*>(&Kc)[i];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int e = blockIdx.x * kAgentWarps + warp;
    if (e >= a.N) return;
    const unsigned FULL = 0xffffffffu;
    const int H = a.H[e], W = a.W[e];
    const int64_t off = a.off[e];
    uint8_t* Fe = a.F + off;
    const uint32_t wmask = W == 32 ? 0xffffffffu : ((1u << W) - 1u);

    // the action: move, valve, water -> this step's drop centre
    int ax = 0, ay = 0, cx = -1, cy = -1;
    if (lane == 0) {
        int act = a.actions[e];
        if (act < 0 || act >= 10) act = 0;
        int x = a.agent[e * 3], y = a.agent[e * 3 + 1], water = a.agent[e * 3 + 2];
        const int move = act % 5;
        if (move == 1) y -= 1;
        if (move == 2) x += 1;
        if (move == 3) y += 1;
        if (move == 4) x -= 1;
        x = min(max(x, 0), W - 1);
        y = min(max(y, 0), H - 1);
        if (act >= 5 && water > 0) {
            cx = x;
            cy = y;
            water -= 1;
        }
        ax = x;
        ay = y;
        a.agent[e * 3] = x;
        a.agent[e * 3 + 1] = y;
        a.agent[e * 3 + 2] = water;
    }
    cx = __shfl_sync(FULL, cx, 0);
    cy = __shfl_sync(FULL, cy, 0);

    uint8_t* buf = s_cells[warp];
    uint32_t B, C, D;
    agent_load_row(Fe, H, W, lane, buf, B, C, D);
    // the tanker drop acts first
    if (cx >= 0 && lane < H && abs(lane - cy) <= a.R) {
        const uint32_t m = bits_between(max(cx - a.R, 0), min(cx + a.R, W - 1));
        const uint32_t doused = B & m;
        B &= ~m;
        D |= doused;
    }
    const int32_t t0 = a.t[e];
    const int32_t ep = a.episode[e];
    const uint32_t tt = (uint32_t)t0, ep4 = 4u * (uint32_t)ep;
    // source masks: the source of direction d for target (y, x) is (y - DR[d], x - DX[d])
    uint32_t Bu = __shfl_up_sync(FULL, B, 1);
    uint32_t Bd = __shfl_down_sync(FULL, B, 1);
    if (lane == 0) Bu = 0u;
    if (lane == 31) Bd = 0u;
    uint32_t sd[8];
    sd[0] = (B << 1) & wmask;
    sd[1] = (Bd << 1) & wmask;
    sd[2] = Bd;
    sd[3] = Bd >> 1;
    sd[4] = B >> 1;
    sd[5] = Bu >> 1;
    sd[6] = Bu;
    sd[7] = (Bu << 1) & wmask;
    const uint32_t cand = C & (sd[0] | sd[1] | sd[2] | sd[3] | sd[4] | sd[5] | sd[6] | sd[7]);
    uint32_t np = 0;
#pragma unroll
    for (int d = 0; d < 8; ++d) np += __popc(sd[d] & cand);
    const int n_items = __popc(B) + (int)(FUSED ? np : __popc(cand));
    int incl = n_items;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(FULL, incl, 31);
    const int excl = incl - n_items;
    s_ig[warp][lane] = 0u;
    s_ou[warp][lane] = 0u;
    __syncwarp();
    for (int pass = 0; pass < total; pass += kAgentList) {
        // items: row << 20 | column << 12 | candidate << 8 | direction or direction mask
        int idx = excl;
        auto put = [&](uint32_t item) {
            if (idx >= pass && idx < pass + kAgentList) s_list[warp][idx - pass] = item;
            ++idx;
        };
        const uint32_t hi = (uint32_t)lane << 20;
        for (uint32_t m = B; m != 0u; m &= m - 1u) put(hi | ((uint32_t)(__ffs(m) - 1) << 12));
        if (FUSED) {
#pragma unroll
            for (int d = 0; d < 8; ++d)
                for (uint32_t m = sd[d] & cand; m != 0u; m &= m - 1u)
                    put(hi | ((uint32_t)(__ffs(m) - 1) << 12) | (1u << 8) | (uint32_t)d);
        } else {
            for (uint32_t m = cand; m != 0u; m &= m - 1u) {
                const int j = __ffs(m) - 1;
                uint32_t dm = 0;
#pragma unroll
                for (int d = 0; d < 8; ++d) dm |= ((sd[d] >> j) & 1u) << d;
                put(hi | ((uint32_t)j << 12) | (1u << 8) | dm);
            }
        }
        __syncwarp();
        const int n_pass = min(kAgentList, total - pass);
        for (int it = lane; it < n_pass; it += 32) {
            const uint32_t item = s_list[warp][it];
            const int yy = (int)(item >> 20), xx = (int)(item >> 12) & 31;
            const bool pair = (item & (1u << 8)) != 0u;
            if (FUSED) {
                const bool below = item_below(a, sK, e, off, W, yy, xx, pair, (int)(item & 7u), tt, ep4);
                if (pair && below) atomicOr(&s_ig[warp][yy], 1u << xx);
                if (!pair && !below) atomicOr(&s_ou[warp][yy], 1u << xx);
            } else {
                const uint32_t cell = (uint32_t)(yy * W + xx);
                if (!pair) {
                    const uint4 u = jwf_philox(make_uint4(cell, tt, (uint32_t)e, ep4 + 2u), a.key0, a.key1);
                    if (!(jwf_u24(u.x) < a.p_continue)) atomicOr(&s_ou[warp][yy], 1u << xx);
                } else if (ignites(a, e, off, cell, item & 0xFFu, tt, ep4)) {
                    atomicOr(&s_ig[warp][yy], 1u << xx);
                }
            }
        }
        __syncwarp();
    }
    const uint32_t ig = s_ig[warp][lane], ou = s_ou[warp][lane];
    B = (B & ~ou) | ig;
    C &= ~ig;
    D |= ou;
    int nburn = __popc(B);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nburn += __shfl_xor_sync(FULL, nburn, o);
    int32_t t = t0 + 1;
    int32_t epn = ep;
    const bool done = (nburn == 0) || (a.t_max > 0 && t >= a.t_max);
    if (lane == 0) {
        if (a.reward) a.reward[e] = -a.burn_penalty * (float)nburn + (nburn == 0 ? 10.0f : 0.0f);
        if (a.done) a.done[e] = done ? 1 : 0;
    }
    if (done && a.auto_reset) {
        // restart: initial state, fresh random stream, the agent somewhere new
        t = 0;
        epn = ep + 1;
        agent_load_row(a.F0 + off, H, W, lane, buf, B, C, D);
        const uint4 w = jwf_philox(make_uint4(0u, 0u, (uint32_t)e, 4u * (uint32_t)epn + 3u), a.key0, a.key1);
        if (lane == 0) {
            ax = min((int)(jwf_u24(w.x) * (float)W), W - 1);
            ay = min((int)(jwf_u24(w.y) * (float)H), H - 1);
            a.agent[e * 3] = ax;
            a.agent[e * 3 + 1] = ay;
            a.agent[e * 3 + 2] = a.water0;
        }
        if (a.random_fire) {
            // the first can-burn cell at or after `start`, row-major, wrapping
            const int n = H * W;
            const int start = min((int)(jwf_u24(w.z) * (float)n), n - 1);
            const int sy = start / W, sx = start - sy * W;
            uint32_t after = 0u;
            if (lane > sy) after = C;
            if (lane == sy) after = C & (sx == 0 ? 0xffffffffu : ~((1u << sx) - 1u));
            uint32_t m1 = __ballot_sync(FULL, after != 0u);
            int hit_lane = -1;
            uint32_t hit_row = 0u;
            if (m1 != 0u) {
                hit_lane = __ffs(m1) - 1;
                hit_row = __shfl_sync(FULL, after, hit_lane);
            } else {
                const uint32_t m2 = __ballot_sync(FULL, C != 0u);
                if (m2 != 0u) {
                    hit_lane = __ffs(m2) - 1;
                    hit_row = __shfl_sync(FULL, C, hit_lane);
                }
            }
            if (hit_lane >= 0 && lane == hit_lane) {
                const uint32_t bit = hit_row & (~hit_row + 1u);       // lowest set bit
                C &= ~bit;
                B |= bit;
            }
        }
    }
    ax = __shfl_sync(FULL, ax, 0);
    ay = __shfl_sync(FULL, ay, 0);
    // state back to memory (rows into the shared buffer, then coalesced stores)
    if (lane < H) {
        uint8_t* row = buf + lane * W;
        for (int x = 0; x < W; ++x)
            row[x] = (uint8_t)(((C >> x) & 1u) + ((B >> x) & 1u) * 2u + ((D >> x) & 1u) * 3u);
    }
    __syncwarp();
    {
        const int n = H * W;
        if ((reinterpret_cast<uintptr_t>(Fe) & 3u) == 0 && (n & 3) == 0) {
            for (int i = lane; i < n / 4; i += 32)
                reinterpret_cast<uint32_t*>(Fe)[i] = reinterpret_cast<const uint32_t*>(buf)[i];
        } else {
            for (int i = lane; i < n; i += 32) Fe[i] = buf[i];
        }
    }
    if (lane == 0) {
        a.t[e] = t;
        a.episode[e] = epn;
    }
    // the egocentric window (255 outside the grid)
    if (a.obs != nullptr) {
        const int k = a.obs_k, r = k / 2;
        for (int i0 = 0; i0 < k * k; i0 += 32) {
            const int i = i0 + lane;
            const int yy = ay - r + i / k, xx = ax - r + i % k;
            const bool inside = i < k * k && yy >= 0 && yy < H && xx >= 0 && xx < W;
            const int src = inside ? yy : 0;
            const uint32_t rb = __shfl_sync(FULL, B, src), rc = __shfl_sync(FULL, C, src), rd = __shfl_sync(FULL, D, src);
            if (i < k * k) {
                uint8_t v = 255;
                if (inside) v = (uint8_t)(((rc >> xx) & 1u) + ((rb >> xx) & 1u) * 2u + ((rd >> xx) & 1u) * 3u);
                a.obs[(int64_t)e * k * k + i] = v;
            }
        }
    }
}

}  // namespace

cudaError_t jwf_launch_agent_warp(const jwf_ctx* c, bool fused, const int32_t* actions, int32_t* agent,
                                  int32_t water0, int random_fire, float burn_penalty, float* reward, uint8_t* done,
                                  int32_t obs_k, uint8_t* obs, cudaStream_t s) {
    AgentArgs a;
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
    a.t = c->d_t;
    a.episode = c->d_episode;
    a.actions = actions;
    a.agent = agent;
    a.reward = reward;
    a.done = done;
    a.obs = obs;
    a.obs_k = obs_k;
    a.t_max = c->t_max;
    a.R = c->drop_radius;
    a.auto_reset = (c->flags & JWF_AUTO_RESET) ? 1 : 0;
    a.water0 = water0;
    a.random_fire = random_fire;
    a.key0 = (uint32_t)(c->seed & 0xffffffffu);
    a.key1 = (uint32_t)(c->seed >> 32);
    a.p_continue = c->P.p_continue;
    a.burn_penalty = burn_penalty;
    RateConsts K;
    if (fused)
        jwf_rate_consts(c, &K);
    else
        K = RateConsts{};
    const unsigned grid = (unsigned)((c->N + kAgentWarps - 1) / kAgentWarps);
    if (fused)
        k_agent_warp<true><<<grid, kAgentWarps * 32, 0, s>>>(a, K);
    else
        k_agent_warp<false><<<grid, kAgentWarps * 32, 0, s>>>(a, K);
    return cudaGetLastError();
}

cudaError_t jwf_launch_agent_act(const jwf_ctx* c, const int32_t* actions, int32_t* agent, cudaStream_t s) {
    k_agent_act<<<(c->N + 255) / 256, 256, 0, s>>>(c->N, c->d_H, c->d_W, actions, agent, c->d_agent_drops);
    return cudaGetLastError();
}

cudaError_t jwf_launch_agent_post(const jwf_ctx* c, int mode, int32_t* agent, int32_t water0, int random_fire,
                                  float burn_penalty, float* reward, int32_t obs_k, uint8_t* obs, cudaStream_t s) {
    k_agent_post<<<(unsigned)c->N, 32, 0, s>>>(
        c->N, c->d_H, c->d_W, c->d_off, c->d_state[c->cur], c->d_episode, c->d_agent_cnt, c->d_agent_done,
        (c->flags & JWF_AUTO_RESET) ? 1 : 0, mode, agent, water0, random_fire, (uint32_t)(c->seed & 0xffffffffu),
        (uint32_t)(c->seed >> 32), burn_penalty, reward, obs_k, obs);
    return cudaGetLastError();
}
