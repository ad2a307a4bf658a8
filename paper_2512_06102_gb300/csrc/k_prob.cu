// k_prob.cu -- per-(cell, direction) ignition tables (Section 3, Eqs. 1-4)
// and their parameter gradient.
//
// k_prob_table: one thread per target cell v computes, for the 8 incoming
// directions d (source u = v - Delta_d),
//   r[v][d] = gamma(v) * phi(u, d),   q[v][d] = 1 - exp(-r[v][d])
// with phi from Eq. 3 (wind Eq. 1 and slope Eq. 2 taken at the source) and
// gamma the target's susceptibility.  HBM-write bound: 32 B of q (and 32 B of
// r) per cell against 5 B of class + elevation read.
//
// k_rates_bwd: dL/dtheta = sum_t sum_{v,d} glam_t(v) pb_t(v - Delta_d) dr[v][d]/dtheta,
// every derivative written without division so that classes with no fuel
// (mu_den = -1) are exact.  Deterministic: per-block FP64 partials, summed in
// a fixed order by the last block to finish.
#include <math.h>

#include <cmath>

#include "jwf_internal.cuh"

namespace {

struct DirConst {
    float cphi[8], sphi[8], inv_len[8];
};

__device__ __forceinline__ DirConst dir_const() {
    const float h = 0.70710678118654752f;   // sqrt(2)/2
    DirConst k = {{1.f, h, 0.f, -h, -1.f, -h, 0.f, h},
                  {0.f, h, 1.f, h, 0.f, -h, -1.f, -h},
                  {1.f, h, 1.f, h, 1.f, h, 1.f, h}};
    return k;
}

// Shape of one directional factor: E = alpha_w1 V + alpha_w2 V (cos - 1) + alpha_s S.
struct RateTerms {
    float S;        // slope in degrees (Eq. 2)
    float cosm1;    // cos(phi_d - Theta) - 1
    float V;        // wind speed at the source
    float K;        // exp(E)
};

__device__ __forceinline__ RateTerms rate_terms(const JwfDevParams& P, float z_src, float z_dst,
                                                float V, float cth, float sth, float cphi,
                                                float sphi, float inv_len, float slope_scale) {
    RateTerms t;
    const float x = (z_dst - z_src) * inv_len;              // rise over run
    t.S = atanf(x) * slope_scale;                           // degrees
    const float cosd = cphi * cth + sphi * sth;             // cos(phi_d - Theta)
    t.cosm1 = cosd - 1.0f;
    t.V = V;
    const float E = P.alpha_w1 * V + P.alpha_w2 * V * t.cosm1 + P.alpha_s * t.S;
    t.K = expf(E);
    return t;
}

// ---------------------------------------------------------------------------
// Double-float helpers (a value is hi + lo with |lo| <= ulp(hi)/2).  Error-free
// transforms use the _rn intrinsics so the compiler cannot contract them.
// ---------------------------------------------------------------------------
struct df {
    float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ df quick_two_sum(float a, float b) {   // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df df_add(df a, df b) {
    const df s = two_sum(a.hi, b.hi);
    return quick_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df df_mul(df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    const float e = fmaf(a.hi, b.hi, -p);
    return quick_two_sum(p, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e)));
}
__device__ __forceinline__ df df_div(df a, df b) {
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const df r = df_add(a, df_neg(df_mul({q1, 0.f}, b)));
    return quick_two_sum(q1, __fdiv_rn(r.hi, b.hi));
}

// Constants prepared on the host in double precision.
struct ProbConsts {
    df atan_th[65];      // theta_k = k pi/256, k = 0..64
    df atan_tan[65];     // tan(theta_k)
    df half_pi;
    df slope_coef;       // alpha_s * 180 / pi: exponent per radian of slope
    df run[8];           // cell_size * |Delta_d|
    float G[16][16];     // gamma(c_v) * p_base (1 + mu_veg(c_u)) (1 + mu_den(c_u)), [c_v][c_u]
};

// atan of a double-float to ~1e-9 absolute: reduce to b = |x| <= 1 (via
// atan(x) = pi/2 - atan(1/x)), pick theta_k near atan(b), and use
// atan(b) = theta_k + atan(u), u = (b - tan theta_k) / (1 + b tan theta_k),
// |u| < 0.012, with atan(u) = u - u^3/3 + u^5/5.
__device__ __forceinline__ df atan_df(df x, const ProbConsts& K) {
    const bool neg = x.hi < 0.f;
    df a = neg ? df_neg(x) : x;
    const bool inv = a.hi > 1.0f;
    const df b = inv ? df_div({1.0f, 0.0f}, a) : a;
    // cheap estimate of atan(b) on [0, 1] (error < 5e-3 rad) to pick the node
    const float est = b.hi / fmaf(0.28f, b.hi * b.hi, 1.0f);
    int k = __float2int_rn(est * 81.48733086305042f);       // 256 / pi
    k = min(max(k, 0), 64);
    const df t = K.atan_tan[k];
    const df num = df_add(b, df_neg(t));
    const df den = df_add({1.0f, 0.0f}, df_mul(b, t));
    const float u = __fdiv_rn(num.hi + num.lo, den.hi);
    const float u2 = u * u;
    const float at_u = u + u * u2 * fmaf(u2, 0.2f, -0.33333334f);
    df th = df_add(K.atan_th[k], {at_u, 0.0f});
    if (inv) th = df_add(K.half_pi, df_neg(th));
    return neg ? df_neg(th) : th;
}

__global__ void k_wind_exponent(int32_t N, const float* __restrict__ ws, const float* __restrict__ wd,
                                double alpha_w1, double alpha_w2, float2* __restrict__ wexp) {
    // alpha_w1 V + alpha_w2 V (cos(d pi/4 - Theta) - 1) per env and direction, in
    // double (cos - 1 written as -2 sin^2 to avoid cancellation), split hi + lo
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N * 8) return;
    const int e = i >> 3, d = i & 7;
    const double V = (double)ws[e], Th = (double)wd[e];
    const double s = sin(0.5 * (d * 0.78539816339744830962 - Th));
    const double w = alpha_w1 * V + alpha_w2 * V * (-2.0 * s * s);
    const float hi = (float)w;
    wexp[i] = make_float2(hi, (float)(w - (double)hi));
}

__global__ void __launch_bounds__(JWF_TILE)
k_prob_table(const int2* __restrict__ tiles, const int32_t* __restrict__ Hs,
             const int32_t* __restrict__ Ws, const int64_t* __restrict__ offs,
             const uint8_t* __restrict__ cls, const float* __restrict__ dem,
             const float* __restrict__ ws, const float* __restrict__ wd,
             const float2* __restrict__ wexp, int per_cell_wind, const JwfDevParams P,
             const ProbConsts K, float* __restrict__ q, float* __restrict__ r) {
    __shared__ ProbConsts sK;
    for (int i = threadIdx.x; i < (int)(sizeof(ProbConsts) / 4); i += blockDim.x)
        reinterpret_cast<float*>(&sK)[i] = reinterpret_cast<const float*>(&K)[i];
    __syncthreads();
    const int2 tile = tiles[blockIdx.x];
    const int e = tile.x;
    const int W = Ws[e], H = Hs[e];
    const int local = tile.y + (int)threadIdx.x;
    if (local >= H * W) return;
    const int64_t off = offs[e];
    const int y = local / W, x = local - (local / W) * W;
    const int64_t v = off + local;

    const int cv = cls[v];
    const float zv = dem[v];
    float rr[8], qq[8];
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        const int uy = y - jwf_dr(d), ux = x - jwf_dx(d);
        rr[d] = 0.f;
        qq[d] = 0.f;
        if (uy < 0 || uy >= H || ux < 0 || ux >= W) continue;
        const int64_t u = off + (int64_t)uy * W + ux;
        const int cu = cls[u];
        const float G = sK.G[cv][cu];
        if (G == 0.f) continue;                      // no fuel at the source or the target
        // wind part of the exponent at the source (Eq. 1)
        df wexp_d;
        if (per_cell_wind) {
            const float V = ws[u];
            const float sn = sinf(0.5f * (d * 0.78539816f - wd[u]));
            wexp_d = {V * fmaf(-2.0f * P.alpha_w2, sn * sn, P.alpha_w1), 0.0f};
        } else {
            const float2 w2 = wexp[e * 8 + d];
            wexp_d = {w2.x, w2.y};
        }
        // slope part (Eq. 2): alpha_s * degrees(atan(dz / run)), in double-float
        const df dz = two_sum(zv, -dem[u]);
        const df slope = atan_df(df_div(dz, sK.run[d]), sK);
        const df E = df_add(wexp_d, df_mul(sK.slope_coef, slope));
        const float kh = expf(E.hi);
        const float kappa = fmaf(kh, E.lo, kh);       // exp(E.hi + E.lo)
        rr[d] = G * kappa;                            // gamma(v) phi(u, d)  (Eqs. 3-4)
        qq[d] = -expm1f(-rr[d]);                      // 1 - exp(-rate)
    }
    float4* q4 = reinterpret_cast<float4*>(q + v * 8);
    q4[0] = make_float4(qq[0], qq[1], qq[2], qq[3]);
    q4[1] = make_float4(qq[4], qq[5], qq[6], qq[7]);
    if (r != nullptr) {
        float4* r4 = reinterpret_cast<float4*>(r + v * 8);
        r4[0] = make_float4(rr[0], rr[1], rr[2], rr[3]);
        r4[1] = make_float4(rr[4], rr[5], rr[6], rr[7]);
    }
}

// ---------------------------------------------------------------------------
// Deterministic block reduction of NV doubles per thread into out[NV]
// (valid in thread 0 .. NV-1 of the block after the call).
// ---------------------------------------------------------------------------
template <int NV>
__device__ void block_reduce_vec(double (&val)[NV], double* smem /* [32][NV] */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        double v = val[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) smem[warp * NV + i] = v;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NV; i += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < nwarps; ++w) s += smem[w * NV + i];
        val[i] = s;
    }
    __syncthreads();
}

constexpr int kRbThreads = 256;
constexpr int kRbScalars = 5;   // p_base, alpha_w1, alpha_w2, alpha_s, alpha_gamma

template <int C>
__global__ void __launch_bounds__(kRbThreads)
k_rates_bwd(const int2* __restrict__ tiles, int64_t n_tiles, const int32_t* __restrict__ Hs,
            const int32_t* __restrict__ Ws, const int64_t* __restrict__ offs, int64_t cells,
            int32_t n_steps, const float* __restrict__ glam, const float* __restrict__ pburn,
            const float* __restrict__ mask, const uint8_t* __restrict__ cls,
            const float* __restrict__ dem, const float* __restrict__ ws,
            const float* __restrict__ wd, int per_cell_wind, const JwfDevParams P,
            double* __restrict__ partials, uint32_t* __restrict__ counter,
            double* __restrict__ gparams) {
    constexpr int NV = kRbScalars + 2 * C;
    __shared__ double red[32 * NV];
    __shared__ bool am_last;
    double acc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = 0.0;
    const DirConst dc = dir_const();
    const float slope_scale = 57.295779513082320876f;
    const float inv_cell = 1.0f / P.cell_size;

    for (int64_t ti = blockIdx.x; ti < n_tiles; ti += gridDim.x) {
        const int2 tile = tiles[ti];
        const int e = tile.x;
        const int W = Ws[e], H = Hs[e];
        const int local = tile.y + (int)threadIdx.x;
        if (local >= H * W) continue;
        const int64_t off = offs[e];
        const int y = local / W, x = local - (local / W) * W;
        const int64_t v = off + local;
        // w[d] = sum_t glam_t(v) * pb_t(v - Delta_d)
        float w[8];
#pragma unroll
        for (int d = 0; d < 8; ++d) w[d] = 0.f;
        for (int t = 0; t < n_steps; ++t) {
            const int64_t base = (int64_t)t * cells;
            const float g = glam[base + v];
            if (g == 0.f) continue;
#pragma unroll
            for (int d = 0; d < 8; ++d) {
                const int uy = y - jwf_dr(d), ux = x - jwf_dx(d);
                if (uy < 0 || uy >= H || ux < 0 || ux >= W) continue;
                const int64_t u = off + (int64_t)uy * W + ux;
                float pb = pburn[base + u];
                if (mask != nullptr) pb *= 1.0f - mask[base + u];
                if (pb != 0.f) w[d] += g * pb;
            }
        }
        const int cv = cls[v];
        const float zv = dem[v];
        const float Av = (1.0f + P.mu_veg[cv]) * (1.0f + P.mu_den[cv]);
        const float gamma = P.alpha_gamma * Av;
        float cth = 0.f, sth = 0.f, Venv = 0.f;
        if (!per_cell_wind) {
            Venv = ws[e];
            sincosf(wd[e], &sth, &cth);
        }
        float g_pb = 0.f, g_w1 = 0.f, g_w2 = 0.f, g_s = 0.f, g_gam = 0.f;
        float tgt = 0.f;        // sum_d w phi: dL/dgamma(v)
        float src[8];           // w * gamma(v) * p_base * K: dL/dA(c_u)
        int cu_d[8];
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            src[d] = 0.f;
            cu_d[d] = -1;
            const int uy = y - jwf_dr(d), ux = x - jwf_dx(d);
            if (uy < 0 || uy >= H || ux < 0 || ux >= W) continue;
            const int64_t u = off + (int64_t)uy * W + ux;
            const int cu = cls[u];
            float V = Venv, c = cth, s = sth;
            if (per_cell_wind) {
                V = ws[u];
                sincosf(wd[u], &s, &c);
            }
            const RateTerms t = rate_terms(P, dem[u], zv, V, c, s, dc.cphi[d], dc.sphi[d],
                                           dc.inv_len[d] * inv_cell, slope_scale);
            const float Au = (1.0f + P.mu_veg[cu]) * (1.0f + P.mu_den[cu]);
            const float phi = P.p_base * Au * t.K;
            const float rate = gamma * phi;
            const float wr = w[d] * rate;
            g_pb += w[d] * gamma * Au * t.K;   // dr/dp_base
            g_w1 += wr * t.V;                  // dr/dalpha_w1
            g_w2 += wr * t.V * t.cosm1;        // dr/dalpha_w2
            g_s += wr * t.S;                   // dr/dalpha_s
            g_gam += w[d] * Av * phi;          // dr/dalpha_gamma
            tgt += w[d] * phi;
            src[d] = w[d] * gamma * P.p_base * t.K;
            cu_d[d] = cu;
        }
        acc[0] += g_pb;
        acc[1] += g_w1;
        acc[2] += g_w2;
        acc[3] += g_s;
        acc[4] += g_gam;
        // mu_veg[k]: target role alpha_gamma (1 + mu_den[k]) tgt; source role (1 + mu_den[k]) src
        // mu_den[k]: target role alpha_gamma (1 + mu_veg[k]) tgt; source role (1 + mu_veg[k]) src
#pragma unroll
        for (int k = 0; k < C; ++k) {
            float sk = 0.f;
#pragma unroll
            for (int d = 0; d < 8; ++d) sk += (cu_d[d] == k) ? src[d] : 0.f;
            const float tk = (cv == k) ? P.alpha_gamma * tgt : 0.f;
            acc[kRbScalars + k] += (double)((tk + sk) * (1.0f + P.mu_den[k]));
            acc[kRbScalars + C + k] += (double)((tk + sk) * (1.0f + P.mu_veg[k]));
        }
    }
    block_reduce_vec<NV>(acc, red);
    if (threadIdx.x < NV) partials[(int64_t)blockIdx.x * NV + threadIdx.x] = acc[threadIdx.x];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) am_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    // the last block sums the block partials in a fixed order
    double tot[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) tot[i] = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
#pragma unroll
        for (int j = 0; j < NV; ++j) tot[j] += __ldcg(&partials[(int64_t)b * NV + j]);
    }
    block_reduce_vec<NV>(tot, red);
    // layout [p_base, alpha_w1, alpha_w2, alpha_s, alpha_gamma, mu_veg[nC], mu_den[nC]]
    const int nC = P.n_classes;
    const int i = threadIdx.x;
    if (i < kRbScalars) {
        gparams[i] += tot[i];
    } else if (i < kRbScalars + C) {
        if (i - kRbScalars < nC) gparams[i] += tot[i];
    } else if (i < NV) {
        const int k = i - kRbScalars - C;
        if (k < nC) gparams[kRbScalars + nC + k] += tot[i];
    }
    if (threadIdx.x == 0) *counter = 0u;
}

template <int C>
cudaError_t launch_rates_bwd_c(jwf_ctx* c, int32_t n_steps, const float* glam,
                               const float* pburn, const float* mask, const uint8_t* cls,
                               const float* dem, const float* ws, const float* wd,
                               double* gparams, cudaStream_t s) {
    constexpr int NV = kRbScalars + 2 * C;
    int64_t grid = (int64_t)c->num_sms * 4;
    if (grid > c->n_tiles) grid = c->n_tiles;
    if (grid * NV > c->partial_cap) grid = c->partial_cap / NV;
    if (grid < 1) return cudaErrorInvalidValue;
    k_rates_bwd<C><<<(unsigned)grid, kRbThreads, 0, s>>>(
        c->d_tiles, c->n_tiles, c->d_H, c->d_W, c->d_off, c->cells, n_steps, glam, pburn, mask,
        cls, dem, ws, wd, (c->flags & JWF_WIND_PER_CELL) ? 1 : 0, c->P, c->d_partials,
        c->d_red_counter, gparams);
    return cudaGetLastError();
}

}  // namespace

static df split_df(double v) {
    const float hi = (float)v;
    return {hi, (float)(v - (double)hi)};
}

cudaError_t jwf_launch_prob_table(const jwf_ctx* c, const uint8_t* cls, const float* dem,
                                  const float* ws, const float* wd, cudaStream_t s) {
    const double pi = 3.14159265358979323846;
    ProbConsts K{};
    for (int k = 0; k <= 64; ++k) {
        const double th = k * pi / 256.0;
        K.atan_th[k] = split_df(th);
        K.atan_tan[k] = split_df(std::tan(th));
    }
    K.half_pi = split_df(pi / 2.0);
    K.slope_coef = split_df((double)c->P.alpha_s * 180.0 / pi);
    for (int d = 0; d < 8; ++d)
        K.run[d] = split_df((double)c->P.cell_size * ((d & 1) ? std::sqrt(2.0) : 1.0));
    for (int a = 0; a < 16; ++a)
        for (int b = 0; b < 16; ++b) {
            if (a >= c->n_classes || b >= c->n_classes) {
                K.G[a][b] = 0.f;
                continue;
            }
            const double gamma = (double)c->P.alpha_gamma * (1.0 + (double)c->P.mu_veg[a]) *
                                 (1.0 + (double)c->P.mu_den[a]);
            const double base = (double)c->P.p_base * (1.0 + (double)c->P.mu_veg[b]) *
                                (1.0 + (double)c->P.mu_den[b]);
            K.G[a][b] = (float)(gamma * base);
        }
    const bool per_cell = (c->flags & JWF_WIND_PER_CELL) != 0u;
    if (!per_cell) {
        k_wind_exponent<<<(c->N * 8 + 255) / 256, 256, 0, s>>>(c->N, ws, wd, (double)c->P.alpha_w1,
                                                                 (double)c->P.alpha_w2, c->d_wexp);
    }
    k_prob_table<<<(unsigned)c->n_tiles, JWF_TILE, 0, s>>>(
        c->d_tiles, c->d_H, c->d_W, c->d_off, cls, dem, ws, wd, c->d_wexp, per_cell ? 1 : 0, c->P, K,
        c->d_q, (c->flags & JWF_KEEP_RATES) ? c->d_r : nullptr);
    return cudaGetLastError();
}

cudaError_t jwf_launch_rates_bwd(jwf_ctx* c, int32_t n_steps, const float* glam,
                                 const float* pburn, const float* mask, const uint8_t* cls,
                                 const float* dem, const float* ws, const float* wd,
                                 double* gparams, cudaStream_t s) {
    // class-count specialisations keep the per-class bins in registers
    const int C = c->n_classes;
    if (C <= 1) return launch_rates_bwd_c<1>(c, n_steps, glam, pburn, mask, cls, dem, ws, wd, gparams, s);
    if (C <= 4) return launch_rates_bwd_c<4>(c, n_steps, glam, pburn, mask, cls, dem, ws, wd, gparams, s);
    if (C <= 11) return launch_rates_bwd_c<11>(c, n_steps, glam, pburn, mask, cls, dem, ws, wd, gparams, s);
    if (C <= 16) return launch_rates_bwd_c<16>(c, n_steps, glam, pburn, mask, cls, dem, ws, wd, gparams, s);
    return cudaErrorNotSupported;
}
