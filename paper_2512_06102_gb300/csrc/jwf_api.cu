// jwf_api.cu -- the C ABI of libjwf (declared in include/jwf.h): argument
// validation, context memory and kernel dispatch.  Every entry point returns a
// jwf_status; nothing here throws, aborts or synchronises unless documented.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>

#include "jwf_internal.cuh"

namespace {

jwf_status fail(jwf_ctx* c, jwf_status st, const char* msg) {
    if (c != nullptr) c->last_error = msg;
    return st;
}

jwf_status cuda_fail(jwf_ctx* c, cudaError_t err, const char* where) {
    if (c != nullptr) {
        c->last_error = std::string(where) + ": " + cudaGetErrorString(err);
    }
    return err == cudaErrorMemoryAllocation ? JWF_ENOMEM : JWF_ECUDA;
}

#define JWF_CUDA_TRY(ctx, expr, where)                           \
    do {                                                         \
        cudaError_t err_ = (expr);                               \
        if (err_ != cudaSuccess) return cuda_fail(ctx, err_, where); \
    } while (0)

template <typename T>
cudaError_t dev_alloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) return cudaSuccess;
    return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
}

void free_all(jwf_ctx* c) {
    for (int g = 0; g < JWF_MAX_GROUPS; ++g) {
        if (c->side[g] != nullptr) cudaStreamDestroy(c->side[g]);
        if (c->ev_join[g] != nullptr) cudaEventDestroy(c->ev_join[g]);
    }
    if (c->ev_fork != nullptr) cudaEventDestroy(c->ev_fork);
    void* ptrs[] = {c->d_H, c->d_W, c->d_off, c->d_order, c->d_tiles, c->d_state[0], c->d_state[1],
                    c->d_F0, c->d_q, c->d_r, c->d_t, c->d_episode, c->d_cnt, c->d_flag,
                    c->d_status, c->d_queue, c->d_partials, c->d_red_counter, c->d_glam, c->d_gr, c->d_wexp,
                    c->d_tiles4, c->d_env_tiles, c->d_tact[0], c->d_tact[1], c->d_tsync, c->d_tburnt,
                    c->d_tcnt, c->d_rtiles, c->d_r2tiles, c->d_adj, c->d_wser, c->d_agent_drops, c->d_agent_cnt,
                    c->d_agent_done, c->d_stiles, c->d_tmaps, c->d_tma_ok, c->d_order_dyn, c->d_lastb,
                    c->d_tplan, c->d_s2tiles, c->d_ptiles};
    for (void* p : ptrs)
        if (p != nullptr) cudaFree(p);
}

inline cudaStream_t S(void* stream) { return reinterpret_cast<cudaStream_t>(stream); }

bool use_resident(const jwf_ctx* c) {
    if (c->kernel == JWF_KERNEL_PLAIN) return false;
    const int threads = c->threads_per_env > 0 ? c->threads_per_env
                                               : jwf_resident_threads(c->maxH, c->maxW);
    const size_t need = jwf_resident_smem(c->maxH, c->maxW, threads);
    int limit = 0;
    cudaDeviceGetAttribute(&limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
    return need + 64 <= (size_t)limit;
}

}  // namespace

extern "C" {

const char* jwf_status_string(jwf_status s) {
    switch (s) {
        case JWF_OK: return "ok";
        case JWF_EINVAL: return "invalid argument";
        case JWF_ENOMEM: return "out of memory";
        case JWF_ECUDA: return "CUDA error";
        case JWF_ETIMEOUT: return "device wait timed out";
        case JWF_ESTATE: return "call out of order";
        case JWF_EUNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char* jwf_last_error(const jwf_ctx* ctx) {
    return ctx == nullptr ? "" : ctx->last_error.c_str();
}

int32_t jwf_n_envs(const jwf_ctx* ctx) { return ctx == nullptr ? 0 : ctx->N; }
int64_t jwf_n_cells(const jwf_ctx* ctx) { return ctx == nullptr ? 0 : ctx->cells; }
int64_t jwf_env_offset(const jwf_ctx* ctx, int32_t e) {
    if (ctx == nullptr || e < 0 || e > ctx->N) return -1;
    return ctx->off[e];
}

jwf_status jwf_create(const jwf_config* cfg, jwf_ctx** out) {
    if (out == nullptr) return JWF_EINVAL;
    *out = nullptr;
    if (cfg == nullptr || cfg->n_envs < 1 || cfg->h_H == nullptr || cfg->h_W == nullptr)
        return JWF_EINVAL;
    if (cfg->n_classes < 1 || cfg->n_classes > 16 || cfg->drop_radius < 0)
        return JWF_EINVAL;
    if ((cfg->flags & ~(JWF_AUTO_RESET | JWF_WIND_PER_CELL | JWF_KEEP_RATES)) != 0u) return JWF_EINVAL;
    const int32_t N = cfg->n_envs;
    for (int32_t e = 0; e < N; ++e) {
        if (cfg->h_H[e] < 1 || cfg->h_W[e] < 1 || cfg->h_H[e] > 65535 || cfg->h_W[e] > 65535)
            return JWF_EINVAL;
        // Philox's cell counter word is 32 bits
        if ((int64_t)cfg->h_H[e] * cfg->h_W[e] > (int64_t)0x7fffffff) return JWF_EINVAL;
    }
    jwf_ctx* c = new (std::nothrow) jwf_ctx();
    if (c == nullptr) return JWF_ENOMEM;
    c->N = N;
    c->n_classes = cfg->n_classes;
    c->seed = cfg->seed;
    c->t_max = cfg->t_max;
    c->drop_radius = cfg->drop_radius;
    c->flags = cfg->flags;
    c->H.assign(cfg->h_H, cfg->h_H + N);
    c->W.assign(cfg->h_W, cfg->h_W + N);
    c->off.resize(N + 1);
    c->off[0] = 0;
    std::vector<int2> tiles;
    for (int32_t e = 0; e < N; ++e) {
        const int64_t n = (int64_t)c->H[e] * c->W[e];
        c->off[e + 1] = c->off[e] + n;
        c->maxH = std::max(c->maxH, c->H[e]);
        c->maxW = std::max(c->maxW, c->W[e]);
        c->max_env_cells = std::max(c->max_env_cells, n);
        for (int64_t s = 0; s < n; s += JWF_TILE) tiles.push_back(make_int2(e, (int)s));
    }
    c->cells = c->off[N];
    c->packed_aligned = true;
    for (int32_t e = 0; e < N; ++e)
        if ((c->off[e] & 31) != 0 || (c->W[e] & 31) != 0) c->packed_aligned = false;
    c->n_tiles = (int64_t)tiles.size();
    std::vector<int2> ptiles;
    for (int32_t e = 0; e < N; ++e) {
        const int64_t nseg = (int64_t)c->H[e] * ((c->W[e] + JWF_PLAIN_SEG - 1) / JWF_PLAIN_SEG);
        for (int64_t s = 0; s < nseg; s += (int64_t)JWF_TILE * JWF_PLAIN_SEGS_PER_THREAD)
            ptiles.push_back(make_int2(e, (int)s));
    }
    c->n_ptiles = (int64_t)ptiles.size();
    // tiles of the tiled path: (env, tile row, tile column) and per-env layout
    std::vector<int4> tiles4, env_tiles(N);
    for (int32_t e = 0; e < N; ++e) {
        const int tr = (c->H[e] + jwf_tile_rows() - 1) / jwf_tile_rows();
        const int tcn = (c->W[e] + jwf_tile_cols() - 1) / jwf_tile_cols();
        env_tiles[e] = make_int4((int)tiles4.size(), tcn, tr, 0);
        for (int r = 0; r < tr; ++r)
            for (int q = 0; q < tcn; ++q) tiles4.push_back(make_int4(e, r, q, 0));
    }
    c->n_tiles4 = (int64_t)tiles4.size();
    // 2-D tiles of the relaxed kernels
    std::vector<int4> rtiles;
    for (int32_t e = 0; e < N; ++e)
        for (int y = 0; y < c->H[e]; y += JWF_RT_ROWS)
            for (int x = 0; x < c->W[e]; x += JWF_RT_COLS) rtiles.push_back(make_int4(e, y, x, 0));
    c->n_rtiles = (int64_t)rtiles.size();
    std::vector<int4> r2tiles;
    for (int32_t e = 0; e < N; ++e)
        for (int y = 0; y < c->H[e]; y += JWF_R2_ROWS)
            for (int x = 0; x < c->W[e]; x += JWF_R2_COLS) r2tiles.push_back(make_int4(e, y, x, 0));
    c->n_r2tiles = (int64_t)r2tiles.size();
    std::vector<int4> stiles;
    for (int32_t e = 0; e < N; ++e)
        for (int y = 0; y < c->H[e]; y += JWF_SW_ROWS)
            for (int x = 0; x < c->W[e]; x += JWF_SW_COLS) stiles.push_back(make_int4(e, y, x, 0));
    c->n_stiles = (int64_t)stiles.size();
    std::vector<int4> s2tiles;
    for (int32_t e = 0; e < N; ++e)
        for (int y = 0; y < c->H[e]; y += JWF_SW2_ROWS)
            for (int x = 0; x < c->W[e]; x += JWF_SW2_COLS) s2tiles.push_back(make_int4(e, y, x, 0));
    c->n_s2tiles = (int64_t)s2tiles.size();
    // processing order: size class (by the longer side) descending, then
    // cells descending; each class is one resident launch
    auto size_class = [&](int32_t e) {
        const int32_t side = std::max(c->H[e], c->W[e]);
        return side <= 64 ? 0 : side <= 128 ? 1 : side <= 256 ? 2 : 3;
    };
    std::vector<int32_t> order(N);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        const int ca = size_class(a), cb = size_class(b);
        if (ca != cb) return ca > cb;
        return (int64_t)c->H[a] * c->W[a] > (int64_t)c->H[b] * c->W[b];
    });
    for (int32_t i = 0; i < N; ++i) {
        const int32_t e = order[i];
        if (c->groups.empty() || c->groups.back().size_class != size_class(e)) {
            JwfGroup G;
            G.start = i;
            G.size_class = size_class(e);
            c->groups.push_back(G);
        }
        JwfGroup& G = c->groups.back();
        G.count += 1;
        G.maxH = std::max(G.maxH, c->H[e]);
        G.maxW = std::max(G.maxW, c->W[e]);
    }

    cudaError_t err = cudaGetDevice(&c->device);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    c->partial_cap = (int64_t)std::max(c->num_sms, 1) * 8 * 40;
    const bool rates = (c->flags & JWF_KEEP_RATES) != 0u;
    if (err == cudaSuccess) err = dev_alloc(&c->d_H, N);
    if (err == cudaSuccess) err = dev_alloc(&c->d_W, N);
    if (err == cudaSuccess) err = dev_alloc(&c->d_off, N + 1);
    if (err == cudaSuccess) err = dev_alloc(&c->d_order, N);
    if (err == cudaSuccess) err = dev_alloc(&c->d_order_dyn, N);
    if (err == cudaSuccess) err = dev_alloc(&c->d_lastb, N);
    if (err == cudaSuccess) err = dev_alloc(&c->d_tiles, tiles.size());
    if (err == cudaSuccess) err = dev_alloc(&c->d_ptiles, ptiles.size());
    if (err == cudaSuccess) err = dev_alloc(&c->d_state[0], (size_t)c->cells);
    if (err == cudaSuccess) err = dev_alloc(&c->d_state[1], (size_t)c->cells);
    if (err == cudaSuccess) err = dev_alloc(&c->d_F0, (size_t)c->cells);
    if (err == cudaSuccess) err = dev_alloc(&c->d_q, (size_t)c->cells * 8);
    if (err == cudaSuccess && rates) err = dev_alloc(&c->d_r, (size_t)c->cells * 8);
    if (err == cudaSuccess && rates) err = dev_alloc(&c->d_glam, (size_t)c->cells);
    if (err == cudaSuccess && rates) err = dev_alloc(&c->d_gr, (size_t)c->cells * 8);
    if (err == cudaSuccess && rates) err = dev_alloc(&c->d_adj, (size_t)c->cells * 2);
    if (err == cudaSuccess) err = dev_alloc(&c->d_rtiles, rtiles.size());
    if (err == cudaSuccess) err = dev_alloc(&c->d_r2tiles, r2tiles.size());
    if (err == cudaSuccess) err = dev_alloc(&c->d_stiles, stiles.size());
    if (err == cudaSuccess) err = dev_alloc(&c->d_s2tiles, s2tiles.size());
    if (err == cudaSuccess) err = dev_alloc(&c->d_agent_drops, 2 * (size_t)N);
    if (err == cudaSuccess) err = dev_alloc(&c->d_agent_cnt, (size_t)N);
    if (err == cudaSuccess) err = dev_alloc(&c->d_agent_done, (size_t)N);
    if (err == cudaSuccess) err = dev_alloc(&c->d_t, N);
    if (err == cudaSuccess) err = dev_alloc(&c->d_episode, N);
    if (err == cudaSuccess) err = dev_alloc(&c->d_cnt, 2 * (size_t)N);
    if (err == cudaSuccess) err = dev_alloc(&c->d_flag, N);
    if (err == cudaSuccess) err = dev_alloc(&c->d_status, 1);
    if (err == cudaSuccess) err = dev_alloc(&c->d_queue, 2 * JWF_MAX_GROUPS);
    if (err == cudaSuccess) err = dev_alloc(&c->d_partials, (size_t)c->partial_cap);
    if (err == cudaSuccess) err = dev_alloc(&c->d_red_counter, 1);
    if (err == cudaSuccess) err = dev_alloc(&c->d_wexp, (size_t)N * 8);
    if (err == cudaSuccess) err = dev_alloc(&c->d_tiles4, tiles4.size());
    if (err == cudaSuccess) err = dev_alloc(&c->d_env_tiles, (size_t)N);
    if (err == cudaSuccess) err = dev_alloc(&c->d_tact[0], tiles4.size());
    if (err == cudaSuccess) err = dev_alloc(&c->d_tact[1], tiles4.size());
    if (err == cudaSuccess) err = dev_alloc(&c->d_tsync, tiles4.size());
    if (err == cudaSuccess) err = dev_alloc(&c->d_tburnt, tiles4.size());
    // two of each: a round's close and the next round's plan run in one launch
    if (err == cudaSuccess) err = dev_alloc(&c->d_tcnt, (size_t)2 * 16 * 2 * N);
    const size_t plan_words = (size_t)4 + N + 2 * tiles4.size();
    if (err == cudaSuccess) err = dev_alloc(&c->d_tplan, 2 * plan_words);
    if (err == cudaSuccess) err = cudaMemset(c->d_tplan, 0, ((size_t)4 + N) * sizeof(int32_t));
    if (err == cudaSuccess) err = cudaMemset(c->d_tplan + plan_words, 0, ((size_t)4 + N) * sizeof(int32_t));
    if (err == cudaSuccess)
        err = cudaMemcpy(c->d_tiles4, tiles4.data(), tiles4.size() * sizeof(int4), cudaMemcpyHostToDevice);
    if (err == cudaSuccess)
        err = cudaMemcpy(c->d_env_tiles, env_tiles.data(), (size_t)N * sizeof(int4), cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemset(c->d_tburnt, 0, tiles4.size() * sizeof(int32_t));
    if (err == cudaSuccess)
        err = cudaMemcpy(c->d_rtiles, rtiles.data(), rtiles.size() * sizeof(int4), cudaMemcpyHostToDevice);
    if (err == cudaSuccess)
        err = cudaMemcpy(c->d_r2tiles, r2tiles.data(), r2tiles.size() * sizeof(int4), cudaMemcpyHostToDevice);
    if (err == cudaSuccess)
        err = cudaMemcpy(c->d_stiles, stiles.data(), stiles.size() * sizeof(int4), cudaMemcpyHostToDevice);
    if (err == cudaSuccess)
        err = cudaMemcpy(c->d_s2tiles, s2tiles.data(), s2tiles.size() * sizeof(int4), cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemcpy(c->d_H, c->H.data(), N * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemcpy(c->d_W, c->W.data(), N * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemcpy(c->d_off, c->off.data(), (N + 1) * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemcpy(c->d_order, order.data(), N * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemcpy(c->d_tiles, tiles.data(), tiles.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (err == cudaSuccess)
        err = cudaMemcpy(c->d_ptiles, ptiles.data(), ptiles.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemset(c->d_t, 0, N * sizeof(int32_t));
    if (err == cudaSuccess) err = cudaMemset(c->d_episode, 0, N * sizeof(int32_t));
    if (err == cudaSuccess) err = cudaMemset(c->d_cnt, 0, 2 * N * sizeof(int32_t));
    if (err == cudaSuccess) err = cudaMemset(c->d_flag, 0, N);
    if (err == cudaSuccess) err = cudaMemset(c->d_status, 0, sizeof(uint32_t));
    if (err == cudaSuccess) err = cudaMemset(c->d_queue, 0, 2 * JWF_MAX_GROUPS * sizeof(uint32_t));
    if (err == cudaSuccess && c->groups.size() > 1) {
        err = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
        for (size_t g = 0; g < c->groups.size() && err == cudaSuccess; ++g) {
            err = cudaStreamCreateWithFlags(&c->side[g], cudaStreamNonBlocking);
            if (err == cudaSuccess) err = cudaEventCreateWithFlags(&c->ev_join[g], cudaEventDisableTiming);
        }
    }
    if (err == cudaSuccess) err = cudaMemset(c->d_red_counter, 0, sizeof(uint32_t));
    if (err == cudaSuccess) err = jwf_build_tile_maps(c);
    if (err == cudaSuccess) err = cudaDeviceSynchronize();
    if (err != cudaSuccess) {
        const jwf_status st = (err == cudaErrorMemoryAllocation) ? JWF_ENOMEM : JWF_ECUDA;
        free_all(c);
        delete c;
        cudaGetLastError();
        return st;
    }
    *out = c;
    return JWF_OK;
}

jwf_status jwf_destroy(jwf_ctx* ctx) {
    if (ctx == nullptr) return JWF_OK;
    const cudaError_t err = cudaDeviceSynchronize();
    free_all(ctx);
    delete ctx;
    return err == cudaSuccess ? JWF_OK : JWF_ECUDA;
}

jwf_status jwf_set_params(jwf_ctx* ctx, const jwf_params* p) {
    if (ctx == nullptr) return JWF_EINVAL;
    if (p == nullptr || p->h_mu_veg == nullptr || p->h_mu_den == nullptr)
        return fail(ctx, JWF_EINVAL, "jwf_set_params: null pointer");
    const float sc[] = {p->p_base, p->alpha_w1, p->alpha_w2, p->alpha_s, p->alpha_gamma, p->p_continue,
                        p->cell_size};
    for (float v : sc)
        if (!std::isfinite(v)) return fail(ctx, JWF_EINVAL, "jwf_set_params: non-finite parameter");
    if (p->p_continue < 0.f || p->p_continue > 1.f)
        return fail(ctx, JWF_EINVAL, "jwf_set_params: p_continue outside [0, 1]");
    if (p->p_base < 0.f || p->alpha_gamma < 0.f || !(p->cell_size > 0.f))
        return fail(ctx, JWF_EINVAL, "jwf_set_params: p_base, alpha_gamma must be >= 0, cell_size > 0");
    for (int k = 0; k < ctx->n_classes; ++k) {
        const float a = p->h_mu_veg[k], b = p->h_mu_den[k];
        if (!(a >= -1.f && a <= 1.f && b >= -1.f && b <= 1.f))
            return fail(ctx, JWF_EINVAL, "jwf_set_params: mu outside [-1, 1]");
    }
    JwfDevParams P{};
    P.p_base = p->p_base;
    P.alpha_w1 = p->alpha_w1;
    P.alpha_w2 = p->alpha_w2;
    P.alpha_s = p->alpha_s;
    P.alpha_gamma = p->alpha_gamma;
    P.p_continue = p->p_continue;
    P.cell_size = p->cell_size;
    P.n_classes = ctx->n_classes;
    for (int k = 0; k < ctx->n_classes; ++k) {
        P.mu_veg[k] = p->h_mu_veg[k];
        P.mu_den[k] = p->h_mu_den[k];
    }
    ctx->P = P;
    ctx->have_params = true;
    ctx->wexp_stale = true;
    ctx->wser_stale = ctx->wser_n > 0;
    return JWF_OK;
}

jwf_status jwf_sync(jwf_ctx* ctx, void* stream) {
    if (ctx == nullptr) return JWF_EINVAL;
    JWF_CUDA_TRY(ctx, cudaStreamSynchronize(S(stream)), "jwf_sync");
    uint32_t st = 0;
    JWF_CUDA_TRY(ctx, cudaMemcpy(&st, ctx->d_status, sizeof(st), cudaMemcpyDeviceToHost), "jwf_sync");
    if (st != 0u) {
        JWF_CUDA_TRY(ctx, cudaMemset(ctx->d_status, 0, sizeof(uint32_t)), "jwf_sync");
        char buf[96];
        std::snprintf(buf, sizeof buf, "device status word 0x%x", st);
        ctx->last_error = buf;
        return JWF_ETIMEOUT;
    }
    return JWF_OK;
}

jwf_status jwf_precompute_probs(jwf_ctx* ctx, const uint8_t* d_class, const float* d_dem,
                                const float* d_wind_speed, const float* d_wind_dir, void* stream) {
    if (ctx == nullptr) return JWF_EINVAL;
    if (!ctx->have_params) return fail(ctx, JWF_ESTATE, "jwf_precompute_probs: no parameters set");
    if (d_class == nullptr || d_dem == nullptr || d_wind_speed == nullptr || d_wind_dir == nullptr)
        return fail(ctx, JWF_EINVAL, "jwf_precompute_probs: null pointer");
    JWF_CUDA_TRY(ctx, jwf_launch_prob_table(ctx, d_class, d_dem, d_wind_speed, d_wind_dir, S(stream)),
                 "jwf_precompute_probs");
    ctx->have_table = true;
    if (!(ctx->flags & JWF_WIND_PER_CELL)) {
        // the table build also left the per-env wind exponent in d_wexp
        ctx->t_cls = d_class;
        ctx->t_dem = d_dem;
        ctx->t_ws = d_wind_speed;
        ctx->t_wd = d_wind_dir;
        ctx->have_terrain = true;
        ctx->wexp_stale = false;
    }
    ctx->have_rates = (ctx->flags & JWF_KEEP_RATES) != 0u;
    return JWF_OK;
}

jwf_status jwf_check_prob_bound(const jwf_ctx* ctx, int64_t n, const uint8_t* d_class_v, const uint8_t* d_class_u,
                                const float* d_z_v, const float* d_z_u, const float* d_wexp, const int32_t* d_dir,
                                float* d_out, void* stream) {
    if (ctx == nullptr) return JWF_EINVAL;
    jwf_ctx* c = const_cast<jwf_ctx*>(ctx);
    if (!ctx->have_params) return fail(c, JWF_ESTATE, "jwf_check_prob_bound: no parameters set");
    if (n < 0) return fail(c, JWF_EINVAL, "jwf_check_prob_bound: n < 0");
    if (n > 0 && (d_class_v == nullptr || d_class_u == nullptr || d_z_v == nullptr || d_z_u == nullptr ||
                  d_wexp == nullptr || d_dir == nullptr || d_out == nullptr))
        return fail(c, JWF_EINVAL, "jwf_check_prob_bound: null pointer");
    JWF_CUDA_TRY(c, jwf_launch_prob_check(ctx, n, d_class_v, d_class_u, d_z_v, d_z_u, d_wexp, d_dir, d_out,
                                          S(stream)),
                 "jwf_check_prob_bound");
    return JWF_OK;
}

jwf_status jwf_set_terrain(jwf_ctx* ctx, const uint8_t* d_class, const float* d_dem,
                           const float* d_wind_speed, const float* d_wind_dir, void* stream) {
    if (ctx == nullptr) return JWF_EINVAL;
    if (!ctx->have_params) return fail(ctx, JWF_ESTATE, "jwf_set_terrain: no parameters set");
    if (d_class == nullptr || d_dem == nullptr || d_wind_speed == nullptr || d_wind_dir == nullptr)
        return fail(ctx, JWF_EINVAL, "jwf_set_terrain: null pointer");
    if (ctx->flags & JWF_WIND_PER_CELL)
        return fail(ctx, JWF_EUNSUPPORTED, "jwf_set_terrain: the fused step takes per-env wind only");
    JWF_CUDA_TRY(ctx, jwf_launch_wind_exponent(ctx, d_wind_speed, d_wind_dir, S(stream)), "jwf_set_terrain");
    ctx->t_cls = d_class;
    ctx->t_dem = d_dem;
    ctx->t_ws = d_wind_speed;
    ctx->t_wd = d_wind_dir;
    ctx->have_terrain = true;
    ctx->wexp_stale = false;
    return JWF_OK;
}

jwf_status jwf_set_wind_series(jwf_ctx* ctx, int32_t n_steps, const float* d_wind_speed,
                               const float* d_wind_dir, void* stream) {
    if (ctx == nullptr) return JWF_EINVAL;
    if (n_steps < 0) return fail(ctx, JWF_EINVAL, "jwf_set_wind_series: n_steps < 0");
    if (n_steps == 0) {
        ctx->wser_n = 0;
        return JWF_OK;
    }
    if (d_wind_speed == nullptr || d_wind_dir == nullptr)
        return fail(ctx, JWF_EINVAL, "jwf_set_wind_series: null pointer");
    if (!ctx->have_params) return fail(ctx, JWF_ESTATE, "jwf_set_wind_series: no parameters set");
    const int64_t need = (int64_t)n_steps * ctx->N * 8;
    if (need > ctx->wser_cap) {
        float2* p = nullptr;
        const cudaError_t err = cudaMalloc(&p, (size_t)need * sizeof(float2));
        if (err != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, err == cudaErrorMemoryAllocation ? JWF_ENOMEM : JWF_ECUDA,
                        "jwf_set_wind_series: allocation failed");
        }
        if (ctx->d_wser != nullptr) {
            cudaStreamSynchronize(S(stream));
            cudaFree(ctx->d_wser);
        }
        ctx->d_wser = p;
        ctx->wser_cap = need;
    }
    ctx->wser_n = n_steps;
    ctx->s_ws = d_wind_speed;
    ctx->s_wd = d_wind_dir;
    JWF_CUDA_TRY(ctx, jwf_launch_wind_series(ctx, S(stream)), "jwf_set_wind_series");
    ctx->wser_stale = false;
    return JWF_OK;
}

jwf_status jwf_set_probs(jwf_ctx* ctx, const float* d_q, const float* d_r, void* stream) {
    if (ctx == nullptr) return JWF_EINVAL;
    if (d_q == nullptr) return fail(ctx, JWF_EINVAL, "jwf_set_probs: d_q is null");
    if (d_r != nullptr && !(ctx->flags & JWF_KEEP_RATES))
        return fail(ctx, JWF_EUNSUPPORTED, "jwf_set_probs: context has no rate table (JWF_KEEP_RATES)");
    const size_t bytes = (size_t)ctx->cells * 8 * sizeof(float);
    JWF_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->d_q, d_q, bytes, cudaMemcpyDeviceToDevice, S(stream)), "jwf_set_probs");
    if (d_r != nullptr) {
        JWF_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->d_r, d_r, bytes, cudaMemcpyDeviceToDevice, S(stream)),
                     "jwf_set_probs");
        ctx->have_rates = true;
    }
    ctx->have_table = true;
    return JWF_OK;
}

jwf_status jwf_get_probs(jwf_ctx* ctx, float** d_q, float** d_r) {
    if (ctx == nullptr) return JWF_EINVAL;
    if (d_q) *d_q = ctx->d_q;
    if (d_r) *d_r = ctx->d_r;
    return JWF_OK;
}

jwf_status jwf_load_state(jwf_ctx* ctx, const uint8_t* d_F0, void* stream) {
    if (ctx == nullptr) return JWF_EINVAL;
    if (d_F0 == nullptr) return fail(ctx, JWF_EINVAL, "jwf_load_state: null pointer");
    ctx->tiles_valid = false;
    JWF_CUDA_TRY(ctx, jwf_launch_load(ctx, d_F0, S(stream)), "jwf_load_state");
    ctx->have_state = true;
    return JWF_OK;
}

jwf_status jwf_load_state_packed(jwf_ctx* ctx, const uint8_t* d_P0, void* stream) {
    if (ctx == nullptr) return JWF_EINVAL;
    if (d_P0 == nullptr) return fail(ctx, JWF_EINVAL, "jwf_load_state_packed: null pointer");
    ctx->tiles_valid = false;
    JWF_CUDA_TRY(ctx, jwf_launch_load_packed(ctx, d_P0, S(stream)), "jwf_load_state_packed");
    ctx->have_state = true;
    return JWF_OK;
}

jwf_status jwf_get_state_packed(jwf_ctx* ctx, uint8_t* d_packed, void* stream) {
    if (ctx == nullptr) return JWF_EINVAL;
    if (d_packed == nullptr) return fail(ctx, JWF_EINVAL, "jwf_get_state_packed: null pointer");
    if (!ctx->have_state) return fail(ctx, JWF_ESTATE, "jwf_get_state_packed: no state loaded");
    JWF_CUDA_TRY(ctx, jwf_launch_pack(ctx->cells, ctx->d_state[ctx->cur], d_packed, S(stream)),
                 "jwf_get_state_packed");
    return JWF_OK;
}

int64_t jwf_packed_size(int64_t n_cells) { return n_cells < 0 ? -1 : jwf_packed_bytes(n_cells); }

jwf_status jwf_pack_states(int64_t n_cells, const uint8_t* d_states, uint8_t* d_packed, void* stream) {
    if (n_cells < 0 || (n_cells > 0 && (d_states == nullptr || d_packed == nullptr))) return JWF_EINVAL;
    return jwf_launch_pack(n_cells, d_states, d_packed, S(stream)) == cudaSuccess ? JWF_OK : JWF_ECUDA;
}

jwf_status jwf_unpack_states(int64_t n_cells, const uint8_t* d_packed, uint8_t* d_states, void* stream) {
    if (n_cells < 0 || (n_cells > 0 && (d_states == nullptr || d_packed == nullptr))) return JWF_EINVAL;
    return jwf_launch_unpack(n_cells, d_packed, d_states, S(stream)) == cudaSuccess ? JWF_OK : JWF_ECUDA;
}

jwf_status jwf_reset(jwf_ctx* ctx, const uint8_t* d_env_mask, void* stream) {
    if (ctx == nullptr) return JWF_EINVAL;
    if (!ctx->have_state) return fail(ctx, JWF_ESTATE, "jwf_reset: no state loaded");
    ctx->tiles_valid = false;
    JWF_CUDA_TRY(ctx, jwf_launch_reset(ctx, d_env_mask, S(stream)), "jwf_reset");
    return JWF_OK;
}

jwf_status jwf_apply_action(jwf_ctx* ctx, const uint8_t* d_mask, void* stream) {
    if (ctx == nullptr) return JWF_EINVAL;
    if (d_mask == nullptr) return fail(ctx, JWF_EINVAL, "jwf_apply_action: null mask");
    if (!ctx->have_state) return fail(ctx, JWF_ESTATE, "jwf_apply_action: no state loaded");
    ctx->tiles_valid = false;
    JWF_CUDA_TRY(ctx, jwf_launch_action(ctx, d_mask, S(stream)), "jwf_apply_action");
    return JWF_OK;
}

jwf_status jwf_step_record(jwf_ctx* ctx, int32_t k, const int32_t* d_drops, int32_t* d_burning,
                           int32_t* d_burnt, uint8_t* d_done, uint8_t* d_history, void* stream) {
    if (ctx == nullptr) return JWF_EINVAL;
    if (d_history == nullptr) return fail(ctx, JWF_EINVAL, "jwf_step_record: d_history is null");
    ctx->hist = d_history;
    ctx->hist_packed = false;
    const jwf_status st = jwf_step(ctx, k, d_drops, d_burning, d_burnt, d_done, stream);
    ctx->hist = nullptr;
    return st;
}

jwf_status jwf_step_record_packed(jwf_ctx* ctx, int32_t k, const int32_t* d_drops, int32_t* d_burning,
                                  int32_t* d_burnt, uint8_t* d_done, uint8_t* d_history, void* stream) {
    if (ctx == nullptr) return JWF_EINVAL;
    if (d_history == nullptr) return fail(ctx, JWF_EINVAL, "jwf_step_record_packed: d_history is null");
    ctx->hist = d_history;
    ctx->hist_packed = true;
    const jwf_status st = jwf_step(ctx, k, d_drops, d_burning, d_burnt, d_done, stream);
    ctx->hist = nullptr;
    ctx->hist_packed = false;
    return st;
}

namespace {
// k steps with the actions as drop centres or as mask bit rows (not both)
jwf_status step_impl(jwf_ctx* ctx, int32_t k, const int32_t* d_drops, const uint32_t* d_masks, int32_t* d_burning,
                     int32_t* d_burnt, uint8_t* d_done, void* stream) {
    if (ctx == nullptr) return JWF_EINVAL;
    if (k < 1) return fail(ctx, JWF_EINVAL, "jwf_step: k < 1");
    if (!ctx->have_params) return fail(ctx, JWF_ESTATE, "jwf_step: no parameters set");
    if (!ctx->have_state) return fail(ctx, JWF_ESTATE, "jwf_step: no state loaded");
    const jwf_kernel kn = ctx->kernel;
    const bool fused = kn == JWF_KERNEL_FUSED || kn == JWF_KERNEL_TILED_FUSED;
    if (fused && !ctx->have_terrain) return fail(ctx, JWF_ESTATE, "jwf_step: fused step needs jwf_set_terrain");
    if (!fused && !ctx->have_table) return fail(ctx, JWF_ESTATE, "jwf_step: no probability table");
    const bool fits = use_resident(ctx);
    if (kn == JWF_KERNEL_RESIDENT && !fits)
        return fail(ctx, JWF_EUNSUPPORTED, "jwf_step: largest env does not fit shared memory");
    bool tiled = kn == JWF_KERNEL_TILED || kn == JWF_KERNEL_TILED_FUSED ||
                 ((kn == JWF_KERNEL_AUTO || kn == JWF_KERNEL_FUSED) && !fits);
    bool plain = kn == JWF_KERNEL_PLAIN;
    if (tiled && (ctx->flags & JWF_AUTO_RESET)) {
        // rounds of several steps cannot restart an env part-way: one launch per step
        if (fused) return fail(ctx, JWF_EUNSUPPORTED, "jwf_step: auto-reset on large grids needs the table");
        tiled = false;
        plain = true;
    }
    if (ctx->wser_n > 0 && !fused)
        return fail(ctx, JWF_EUNSUPPORTED, "jwf_step: a wind series needs a fused kernel (rates from the terrain)");
    if (fused && ctx->wser_n > 0 && ctx->wser_stale) {
        JWF_CUDA_TRY(ctx, jwf_launch_wind_series(ctx, S(stream)), "jwf_step");
        ctx->wser_stale = false;
    }
    cudaError_t err;
    if (fused && ctx->wexp_stale) {
        JWF_CUDA_TRY(ctx, jwf_launch_wind_exponent(ctx, ctx->t_ws, ctx->t_wd, S(stream)), "jwf_step");
        ctx->wexp_stale = false;
    }
    if (tiled) {
        err = jwf_launch_step_tiled(ctx, k, d_drops, d_masks, d_burning, d_burnt, d_done, fused, S(stream));
    } else {
        ctx->tiles_valid = false;
        if (plain)
            err = jwf_launch_step_plain(ctx, k, d_drops, d_masks, d_burning, d_burnt, d_done, S(stream));
        else
            err = jwf_launch_step_resident(ctx, k, d_drops, d_masks, d_burning, d_burnt, d_done, S(stream));
    }
    if (err != cudaSuccess) return cuda_fail(ctx, err, "jwf_step");
    return JWF_OK;
}
}  // namespace

jwf_status jwf_step(jwf_ctx* ctx, int32_t k, const int32_t* d_drops, int32_t* d_burning,
                    int32_t* d_burnt, uint8_t* d_done, void* stream) {
    return step_impl(ctx, k, d_drops, nullptr, d_burning, d_burnt, d_done, stream);
}

jwf_status jwf_step_masked(jwf_ctx* ctx, int32_t k, const uint32_t* d_mask_bits, int32_t* d_burning,
                           int32_t* d_burnt, uint8_t* d_done, void* stream) {
    if (ctx == nullptr) return JWF_EINVAL;
    if (d_mask_bits == nullptr) return fail(ctx, JWF_EINVAL, "jwf_step_masked: d_mask_bits is null");
    return step_impl(ctx, k, nullptr, d_mask_bits, d_burning, d_burnt, d_done, stream);
}

int64_t jwf_mask_words(int64_t n_cells) { return n_cells < 0 ? 0 : jwf_mask_row_words(n_cells); }

jwf_status jwf_pack_masks(int32_t n_rows, int64_t n_cells, const uint8_t* d_masks, uint32_t* d_bits,
                          void* stream) {
    if (n_rows < 0 || n_cells < 0) return JWF_EINVAL;
    if (n_rows == 0 || n_cells == 0) return JWF_OK;
    if (d_masks == nullptr || d_bits == nullptr) return JWF_EINVAL;
    return jwf_launch_pack_masks(n_rows, n_cells, d_masks, d_bits, S(stream)) == cudaSuccess ? JWF_OK : JWF_ECUDA;
}

namespace {
jwf_status agent_args(jwf_ctx* ctx, const char* who, int32_t* d_agent, int32_t water0, int32_t obs_k, uint8_t* d_obs) {
    if (d_agent == nullptr) return fail(ctx, JWF_EINVAL, who);
    if (water0 < 0) return fail(ctx, JWF_EINVAL, who);
    if (d_obs != nullptr && (obs_k < 1 || obs_k > 63 || obs_k % 2 == 0)) return fail(ctx, JWF_EINVAL, who);
    return JWF_OK;
}
}  // namespace

jwf_status jwf_agent_reset(jwf_ctx* ctx, int32_t* d_agent, int32_t water0, int32_t random_fire, int32_t obs_k,
                           uint8_t* d_obs, void* stream) {
    if (ctx == nullptr) return JWF_EINVAL;
    const jwf_status st = agent_args(ctx, "jwf_agent_reset: bad argument", d_agent, water0, obs_k, d_obs);
    if (st != JWF_OK) return st;
    if (!ctx->have_state) return fail(ctx, JWF_ESTATE, "jwf_agent_reset: no state loaded");
    JWF_CUDA_TRY(ctx, jwf_launch_agent_post(ctx, 1, d_agent, water0, random_fire ? 1 : 0, 0.0f, nullptr, obs_k,
                                            d_obs, S(stream)),
                 "jwf_agent_reset");
    ctx->tiles_valid = false;
    return JWF_OK;
}

jwf_status jwf_agent_step(jwf_ctx* ctx, const int32_t* d_actions, int32_t* d_agent, int32_t water0,
                          int32_t random_fire, float burn_penalty, float* d_reward, uint8_t* d_done, int32_t obs_k,
                          uint8_t* d_obs, void* stream) {
    if (ctx == nullptr) return JWF_EINVAL;
    if (d_actions == nullptr) return fail(ctx, JWF_EINVAL, "jwf_agent_step: d_actions is null");
    const jwf_status st = agent_args(ctx, "jwf_agent_step: bad argument", d_agent, water0, obs_k, d_obs);
    if (st != JWF_OK) return st;
    const jwf_kernel kn = ctx->kernel;
    if (ctx->maxH <= 32 && ctx->maxW <= 32 && ctx->have_state &&
        (kn == JWF_KERNEL_AUTO || kn == JWF_KERNEL_RESIDENT || kn == JWF_KERNEL_FUSED)) {
        // grids of at most 32 x 32: the whole agent step in one warp-per-env launch
        const bool fused = kn == JWF_KERNEL_FUSED;
        if (!ctx->have_params) return fail(ctx, JWF_ESTATE, "jwf_agent_step: no parameters set");
        if (fused && !ctx->have_terrain) return fail(ctx, JWF_ESTATE, "jwf_agent_step: fused step needs terrain");
        if (!fused && !ctx->have_table) return fail(ctx, JWF_ESTATE, "jwf_agent_step: no probability table");
        if (ctx->wser_n > 0 && !fused)
            return fail(ctx, JWF_EUNSUPPORTED, "jwf_agent_step: a wind series needs the fused kernel");
        if (fused && ctx->wser_n > 0 && ctx->wser_stale) {
            JWF_CUDA_TRY(ctx, jwf_launch_wind_series(ctx, S(stream)), "jwf_agent_step");
            ctx->wser_stale = false;
        }
        if (fused && ctx->wexp_stale) {
            JWF_CUDA_TRY(ctx, jwf_launch_wind_exponent(ctx, ctx->t_ws, ctx->t_wd, S(stream)), "jwf_agent_step");
            ctx->wexp_stale = false;
        }
        JWF_CUDA_TRY(ctx, jwf_launch_agent_warp(ctx, fused, d_actions, d_agent, water0, random_fire ? 1 : 0,
                                                burn_penalty, d_reward, d_done, obs_k, d_obs, S(stream)),
                     "jwf_agent_step");
        ctx->tiles_valid = false;
        return JWF_OK;
    }
    JWF_CUDA_TRY(ctx, jwf_launch_agent_act(ctx, d_actions, d_agent, S(stream)), "jwf_agent_step");
    const jwf_status ss = jwf_step(ctx, 1, ctx->d_agent_drops, ctx->d_agent_cnt, nullptr, ctx->d_agent_done, stream);
    if (ss != JWF_OK) return ss;
    JWF_CUDA_TRY(ctx, jwf_launch_agent_post(ctx, 0, d_agent, water0, random_fire ? 1 : 0, burn_penalty, d_reward,
                                            obs_k, d_obs, S(stream)),
                 "jwf_agent_step");
    if (d_done != nullptr)
        JWF_CUDA_TRY(ctx, cudaMemcpyAsync(d_done, ctx->d_agent_done, (size_t)ctx->N, cudaMemcpyDeviceToDevice,
                                          S(stream)),
                     "jwf_agent_step");
    ctx->tiles_valid = false;
    return JWF_OK;
}

jwf_status jwf_set_seed(jwf_ctx* ctx, uint64_t seed) {
    if (ctx == nullptr) return JWF_EINVAL;
    ctx->seed = seed;
    return JWF_OK;
}

jwf_status jwf_state_planes(jwf_ctx* ctx, int32_t n, const uint8_t* d_states, float* d_pun, float* d_pburn,
                            void* stream) {
    if (ctx == nullptr) return JWF_EINVAL;
    if (n < 0) return fail(ctx, JWF_EINVAL, "jwf_state_planes: n < 0");
    if (d_states == nullptr || d_pun == nullptr || d_pburn == nullptr)
        return fail(ctx, JWF_EINVAL, "jwf_state_planes: null pointer");
    if (n == 0) return JWF_OK;
    JWF_CUDA_TRY(ctx, jwf_launch_state_planes((int64_t)n * ctx->cells, d_states, d_pun, d_pburn, S(stream)),
                 "jwf_state_planes");
    return JWF_OK;
}

jwf_status jwf_set_kernel(jwf_ctx* ctx, jwf_kernel kernel, int32_t threads_per_env) {
    if (ctx == nullptr) return JWF_EINVAL;
    if ((int)kernel < (int)JWF_KERNEL_AUTO || (int)kernel > (int)JWF_KERNEL_TILED_FUSED)
        return fail(ctx, JWF_EINVAL, "jwf_set_kernel: unknown kernel");
    const bool tiled = kernel == JWF_KERNEL_TILED || kernel == JWF_KERNEL_TILED_FUSED;
    const int t = threads_per_env;
    if (tiled && !(t == 0 || t == 128 || t == 256 || t == 512))
        return fail(ctx, JWF_EINVAL, "jwf_set_kernel: tiled kernels take 0, 128, 256 or 512 threads a tile");
    if (!tiled && !(t == 0 || t == 32 || t == 64 || t == 128 || t == 256 || t == 512 || t == 1024))
        return fail(ctx, JWF_EINVAL, "jwf_set_kernel: threads_per_env must be 0, 32, 64, 128, 256, 512 or 1024");
    ctx->kernel = kernel;
    ctx->threads_per_env = threads_per_env;
    return JWF_OK;
}

jwf_status jwf_set_class_threads(jwf_ctx* ctx, int32_t size_class, int32_t threads) {
    if (ctx == nullptr) return JWF_EINVAL;
    if (size_class < 0 || size_class > 3) return fail(ctx, JWF_EINVAL, "jwf_set_class_threads: class must be 0..3");
    if (threads != 0 && threads != 32 && threads != 64 && threads != 128 && threads != 256 && threads != 512 &&
        threads != 1024)
        return fail(ctx, JWF_EINVAL, "jwf_set_class_threads: threads must be 0, 32, 64, 128, 256, 512 or 1024");
    int limit = 0;
    cudaDeviceGetAttribute(&limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
    for (const JwfGroup& G : ctx->groups)
        if (G.size_class == size_class && threads > 0 &&
            jwf_resident_smem(G.maxH, G.maxW, threads) + 64 > (size_t)limit)
            return fail(ctx, JWF_EINVAL, "jwf_set_class_threads: the class's envs and that block size do not fit "
                                         "shared memory");
    for (JwfGroup& G : ctx->groups)
        if (G.size_class == size_class) G.threads = threads;
    return JWF_OK;
}

jwf_status jwf_set_env_priority(jwf_ctx* ctx, const float* h_priority) {
    if (ctx == nullptr) return JWF_EINVAL;
    std::vector<int32_t> order(ctx->N);
    JWF_CUDA_TRY(ctx, cudaMemcpy(order.data(), ctx->d_order, ctx->N * sizeof(int32_t), cudaMemcpyDeviceToHost),
                 "jwf_set_env_priority");
    for (const JwfGroup& G : ctx->groups) {
        auto b = order.begin() + G.start, e = b + G.count;
        if (h_priority == nullptr) {
            // back to the creation order: cells descending, then env index
            std::stable_sort(b, e, [&](int32_t x, int32_t y) { return x < y; });
            std::stable_sort(b, e, [&](int32_t x, int32_t y) {
                return (int64_t)ctx->H[x] * ctx->W[x] > (int64_t)ctx->H[y] * ctx->W[y];
            });
        } else {
            std::stable_sort(b, e, [&](int32_t x, int32_t y) { return h_priority[x] > h_priority[y]; });
        }
    }
    JWF_CUDA_TRY(ctx, cudaMemcpy(ctx->d_order, order.data(), ctx->N * sizeof(int32_t), cudaMemcpyHostToDevice),
                 "jwf_set_env_priority");
    return JWF_OK;
}

jwf_status jwf_set_reorder_steps(jwf_ctx* ctx, int32_t steps) {
    if (ctx == nullptr) return JWF_EINVAL;
    if (steps < 0) return fail(ctx, JWF_EINVAL, "jwf_set_reorder_steps: steps < 0");
    ctx->reorder_steps = steps;
    return JWF_OK;
}

jwf_status jwf_set_tile_copy(jwf_ctx* ctx, int32_t tma) {
    if (ctx == nullptr) return JWF_EINVAL;
    if (tma != 0 && tma != 1) return fail(ctx, JWF_EINVAL, "jwf_set_tile_copy: mode must be 0 or 1");
    if (tma == 1 && !ctx->tma) return fail(ctx, JWF_EUNSUPPORTED, "jwf_set_tile_copy: no env qualifies for TMA");
    ctx->use_tma = tma == 1;
    return JWF_OK;
}

jwf_status jwf_set_tile_copy_wait(jwf_ctx* ctx, uint64_t timeout_ns, int32_t no_copy) {
    if (ctx == nullptr) return JWF_EINVAL;
    if (timeout_ns == 0 || timeout_ns > 10000000000ull)
        return fail(ctx, JWF_EINVAL, "jwf_set_tile_copy_wait: timeout must be 1 ns .. 10 s");
    ctx->tma_wait_ns = timeout_ns;
    ctx->tma_diag_no_copy = no_copy != 0;
    return JWF_OK;
}

int32_t jwf_tile_copy(const jwf_ctx* ctx) { return ctx != nullptr && ctx->tma && ctx->use_tma ? 1 : 0; }

jwf_status jwf_set_round_steps(jwf_ctx* ctx, int32_t steps) {
    if (ctx == nullptr) return JWF_EINVAL;
    if (steps < 1 || steps > 16) return fail(ctx, JWF_EINVAL, "jwf_set_round_steps: steps must be 1..16");
    ctx->round_steps = steps;
    return JWF_OK;
}

int32_t jwf_size_classes(const jwf_ctx* ctx, int32_t* h_classes) {
    if (ctx == nullptr) return 0;
    for (size_t g = 0; g < ctx->groups.size(); ++g)
        if (h_classes != nullptr) h_classes[g] = ctx->groups[g].size_class;
    return (int32_t)ctx->groups.size();
}

jwf_status jwf_set_pair_counter(jwf_ctx* ctx, unsigned long long* d_pairs) {
    if (ctx == nullptr) return JWF_EINVAL;
    ctx->d_pairs = d_pairs;
    return JWF_OK;
}

jwf_status jwf_get_state(jwf_ctx* ctx, uint8_t** d_state, int32_t** d_t, int32_t** d_episode) {
    if (ctx == nullptr) return JWF_EINVAL;
    if (d_state) *d_state = ctx->d_state[ctx->cur];
    if (d_t) *d_t = ctx->d_t;
    if (d_episode) *d_episode = ctx->d_episode;
    return JWF_OK;
}

jwf_status jwf_set_relaxed_kernel(jwf_ctx* ctx, int32_t kernel) {
    if (ctx == nullptr) return JWF_EINVAL;
    if (kernel != JWF_RELAXED_TILED && kernel != JWF_RELAXED_PLAIN)
        return fail(ctx, JWF_EINVAL, "jwf_set_relaxed_kernel: unknown kernel");
    ctx->relaxed_kernel = kernel;
    return JWF_OK;
}

jwf_status jwf_step_relaxed_fwd(jwf_ctx* ctx, const float* d_pun, const float* d_pburn,
                                const float* d_mask, float* d_pun_out, float* d_pburn_out,
                                void* stream) {
    if (ctx == nullptr) return JWF_EINVAL;
    if (d_pun == nullptr || d_pburn == nullptr || d_pun_out == nullptr || d_pburn_out == nullptr)
        return fail(ctx, JWF_EINVAL, "jwf_step_relaxed_fwd: null pointer");
    if (d_pun_out == d_pun || d_pun_out == d_pburn || d_pburn_out == d_pun || d_pburn_out == d_pburn)
        return fail(ctx, JWF_EINVAL, "jwf_step_relaxed_fwd: outputs alias inputs");
    if (!ctx->have_params || !ctx->have_rates)
        return fail(ctx, JWF_ESTATE, "jwf_step_relaxed_fwd: needs parameters and a rate table");
    JWF_CUDA_TRY(ctx, jwf_launch_relaxed_fwd(ctx, d_pun, d_pburn, d_mask, d_pun_out, d_pburn_out, S(stream)),
                 "jwf_step_relaxed_fwd");
    return JWF_OK;
}

jwf_status jwf_step_relaxed_bwd(jwf_ctx* ctx, const float* d_pun, const float* d_pburn,
                                const float* d_mask, const float* d_gun_out,
                                const float* d_gburn_out, float* d_gun, float* d_gburn,
                                float* d_glam, double* d_gpc, void* stream) {
    if (ctx == nullptr) return JWF_EINVAL;
    if (d_pun == nullptr || d_pburn == nullptr || d_gun_out == nullptr || d_gburn_out == nullptr ||
        d_gun == nullptr || d_gburn == nullptr)
        return fail(ctx, JWF_EINVAL, "jwf_step_relaxed_bwd: null pointer");
    const void* ins[] = {d_pun, d_pburn, d_mask, d_gun_out, d_gburn_out};
    const void* outs[] = {d_gun, d_gburn, d_glam};
    for (const void* o : outs)
        for (const void* i : ins)
            if (o != nullptr && o == i) return fail(ctx, JWF_EINVAL, "jwf_step_relaxed_bwd: outputs alias inputs");
    if (!ctx->have_params || !ctx->have_rates)
        return fail(ctx, JWF_ESTATE, "jwf_step_relaxed_bwd: needs parameters and a rate table");
    float* glam = d_glam != nullptr ? d_glam : ctx->d_glam;
    JWF_CUDA_TRY(ctx, jwf_launch_relaxed_bwd(ctx, d_pun, d_pburn, d_mask, d_gun_out, d_gburn_out, d_gun, d_gburn,
                                             glam, d_gpc, S(stream)),
                 "jwf_step_relaxed_bwd");
    return JWF_OK;
}

namespace {
// [p, p + n) and [q, q + m) overlap (element counts)
bool overlap(const float* p, int64_t n, const float* q, int64_t m) {
    return p != nullptr && q != nullptr && p < q + m && q < p + n;
}
}  // namespace

jwf_status jwf_relaxed_fwd_steps(jwf_ctx* ctx, int32_t n_steps, const float* d_pun, const float* d_pburn,
                                 const float* d_masks, float* d_pun_out, float* d_pburn_out, void* stream) {
    if (ctx == nullptr) return JWF_EINVAL;
    if (n_steps < 0) return fail(ctx, JWF_EINVAL, "jwf_relaxed_fwd_steps: n_steps < 0");
    if (d_pun == nullptr || d_pburn == nullptr || d_pun_out == nullptr || d_pburn_out == nullptr)
        return fail(ctx, JWF_EINVAL, "jwf_relaxed_fwd_steps: null pointer");
    const int64_t C = ctx->cells, nC = (int64_t)n_steps * C;
    if (overlap(d_pun_out, nC, d_pun, C) || overlap(d_pun_out, nC, d_pburn, C) ||
        overlap(d_pburn_out, nC, d_pun, C) || overlap(d_pburn_out, nC, d_pburn, C) ||
        overlap(d_pun_out, nC, d_pburn_out, nC))
        return fail(ctx, JWF_EINVAL, "jwf_relaxed_fwd_steps: outputs overlap inputs");
    if (!ctx->have_params || !ctx->have_rates)
        return fail(ctx, JWF_ESTATE, "jwf_relaxed_fwd_steps: needs parameters and a rate table");
    for (int32_t t = 0; t < n_steps;) {
        const float* iu = t == 0 ? d_pun : d_pun_out + (t - 1) * C;
        const float* ib = t == 0 ? d_pburn : d_pburn_out + (t - 1) * C;
        const float* m = d_masks != nullptr ? d_masks + (int64_t)t * C : nullptr;
        if (t + 1 < n_steps && ctx->relaxed_kernel == JWF_RELAXED_TILED) {
            // two steps per pass: the rate rows are read once for both
            JWF_CUDA_TRY(ctx,
                         jwf_launch_relaxed_fwd2(ctx, iu, ib, m, m != nullptr ? m + C : nullptr, d_pun_out + t * C,
                                                 d_pburn_out + t * C, d_pun_out + (t + 1) * C,
                                                 d_pburn_out + (t + 1) * C, S(stream)),
                         "jwf_relaxed_fwd_steps");
            t += 2;
        } else {
            JWF_CUDA_TRY(ctx,
                         jwf_launch_relaxed_fwd(ctx, iu, ib, m, d_pun_out + t * C, d_pburn_out + t * C, S(stream)),
                         "jwf_relaxed_fwd_steps");
            t += 1;
        }
    }
    return JWF_OK;
}

jwf_status jwf_relaxed_bwd_steps(jwf_ctx* ctx, int32_t n_steps, const float* d_pun, const float* d_pburn,
                                 const float* d_masks, const float* d_gun_out, const float* d_gburn_out,
                                 float* d_gun, float* d_gburn, float* d_glam, double* d_gpc, void* stream) {
    if (ctx == nullptr) return JWF_EINVAL;
    if (n_steps < 1) return fail(ctx, JWF_EINVAL, "jwf_relaxed_bwd_steps: n_steps < 1");
    if (d_pun == nullptr || d_pburn == nullptr || d_gun_out == nullptr || d_gburn_out == nullptr ||
        d_gun == nullptr || d_gburn == nullptr)
        return fail(ctx, JWF_EINVAL, "jwf_relaxed_bwd_steps: null pointer");
    if (ctx->d_adj == nullptr) return fail(ctx, JWF_EUNSUPPORTED, "jwf_relaxed_bwd_steps: needs JWF_KEEP_RATES");
    const int64_t C = ctx->cells, nC = (int64_t)n_steps * C;
    const float* outs[] = {d_gun, d_gburn};
    for (const float* o : outs)
        if (overlap(o, C, d_pun, nC) || overlap(o, C, d_pburn, nC) || overlap(o, C, d_masks, nC) ||
            overlap(o, C, d_gun_out, C) || overlap(o, C, d_gburn_out, C) || overlap(o, C, d_glam, nC))
            return fail(ctx, JWF_EINVAL, "jwf_relaxed_bwd_steps: outputs overlap inputs");
    if (overlap(d_gun, C, d_gburn, C) || overlap(d_glam, nC, d_pun, nC) || overlap(d_glam, nC, d_pburn, nC) ||
        overlap(d_glam, nC, d_gun_out, C) || overlap(d_glam, nC, d_gburn_out, C))
        return fail(ctx, JWF_EINVAL, "jwf_relaxed_bwd_steps: outputs overlap inputs");
    if (!ctx->have_params || !ctx->have_rates)
        return fail(ctx, JWF_ESTATE, "jwf_relaxed_bwd_steps: needs parameters and a rate table");
    // passes from the last step down: one step (an odd count's last step, or
    // every step on the plain kernels) or two (the tiled kernels); the passes
    // alternate between the outputs and the context's scratch so that the
    // last pass, the one that ends at step 0, writes the outputs
    const bool two = ctx->relaxed_kernel == JWF_RELAXED_TILED && d_glam != nullptr;
    const int32_t passes = two ? n_steps / 2 + n_steps % 2 : n_steps;
    float* su = ctx->d_adj;
    float* sb = ctx->d_adj + C;
    const float* iu = d_gun_out;
    const float* ib = d_gburn_out;
    int32_t t_hi = n_steps;               // the pass covers steps [t_lo, t_hi)
    for (int32_t p = 0; p < passes; ++p) {
        const int32_t len = (two && !(p == 0 && n_steps % 2 == 1)) ? 2 : 1;
        const int32_t t = t_hi - len;
        const bool to_out = (passes - 1 - p) % 2 == 0;
        float* ou = to_out ? d_gun : su;
        float* ob = to_out ? d_gburn : sb;
        const float* m = d_masks != nullptr ? d_masks + (int64_t)t * C : nullptr;
        if (len == 2) {
            JWF_CUDA_TRY(ctx,
                         jwf_launch_relaxed_bwd2(ctx, d_pun + t * C, d_pburn + t * C, m, d_pun + (t + 1) * C,
                                                 d_pburn + (t + 1) * C, m != nullptr ? m + C : nullptr, iu, ib, ou,
                                                 ob, d_glam + (int64_t)t * C, d_glam + (int64_t)(t + 1) * C, d_gpc,
                                                 S(stream)),
                         "jwf_relaxed_bwd_steps");
        } else {
            float* glam = d_glam != nullptr ? d_glam + (int64_t)t * C : ctx->d_glam;
            JWF_CUDA_TRY(ctx, jwf_launch_relaxed_bwd(ctx, d_pun + t * C, d_pburn + t * C, m, iu, ib, ou, ob, glam,
                                                     d_gpc, S(stream)),
                         "jwf_relaxed_bwd_steps");
        }
        iu = ou;
        ib = ob;
        t_hi = t;
    }
    return JWF_OK;
}

jwf_status jwf_rates_accumulate(jwf_ctx* ctx, int32_t n_steps, const float* d_glam, const float* d_pburn,
                                const float* d_mask, float* d_gr, void* stream) {
    if (ctx == nullptr) return JWF_EINVAL;
    if (n_steps < 0) return fail(ctx, JWF_EINVAL, "jwf_rates_accumulate: n_steps < 0");
    if (d_glam == nullptr || d_pburn == nullptr || d_gr == nullptr)
        return fail(ctx, JWF_EINVAL, "jwf_rates_accumulate: null pointer");
    if (n_steps == 0) return JWF_OK;
    JWF_CUDA_TRY(ctx, jwf_launch_rates_accumulate(ctx, n_steps, d_glam, d_pburn, d_mask, d_gr, S(stream)),
                 "jwf_rates_accumulate");
    return JWF_OK;
}

jwf_status jwf_rates_contract(jwf_ctx* ctx, const float* d_gr, const uint8_t* d_class, const float* d_dem,
                              const float* d_wind_speed, const float* d_wind_dir, double* d_gparams,
                              void* stream) {
    if (ctx == nullptr) return JWF_EINVAL;
    if (d_gr == nullptr || d_class == nullptr || d_dem == nullptr || d_wind_speed == nullptr ||
        d_wind_dir == nullptr || d_gparams == nullptr)
        return fail(ctx, JWF_EINVAL, "jwf_rates_contract: null pointer");
    if (!ctx->have_params) return fail(ctx, JWF_ESTATE, "jwf_rates_contract: no parameters set");
    JWF_CUDA_TRY(ctx, jwf_launch_rates_contract(ctx, d_gr, d_class, d_dem, d_wind_speed, d_wind_dir, d_gparams,
                                                S(stream)),
                 "jwf_rates_contract");
    return JWF_OK;
}

jwf_status jwf_rates_bwd(jwf_ctx* ctx, int32_t n_steps, const float* d_glam,
                         const float* d_pburn, const float* d_mask, const uint8_t* d_class,
                         const float* d_dem, const float* d_wind_speed,
                         const float* d_wind_dir, double* d_gparams, void* stream) {
    if (ctx == nullptr) return JWF_EINVAL;
    if (n_steps < 0) return fail(ctx, JWF_EINVAL, "jwf_rates_bwd: n_steps < 0");
    if (d_glam == nullptr || d_pburn == nullptr || d_class == nullptr || d_dem == nullptr ||
        d_wind_speed == nullptr || d_wind_dir == nullptr || d_gparams == nullptr)
        return fail(ctx, JWF_EINVAL, "jwf_rates_bwd: null pointer");
    if (!ctx->have_params) return fail(ctx, JWF_ESTATE, "jwf_rates_bwd: no parameters set");
    if (ctx->d_gr == nullptr) return fail(ctx, JWF_EUNSUPPORTED, "jwf_rates_bwd: needs JWF_KEEP_RATES");
    if (n_steps == 0) return JWF_OK;
    JWF_CUDA_TRY(ctx, jwf_launch_rates_bwd(ctx, n_steps, d_glam, d_pburn, d_mask, d_class, d_dem, d_wind_speed,
                                           d_wind_dir, d_gparams, S(stream)),
                 "jwf_rates_bwd");
    return JWF_OK;
}

}  // extern "C"
