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
#include "jwf_internal.cuh"

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

}  // namespace

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
