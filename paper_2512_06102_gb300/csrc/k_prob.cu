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
#include "rate_model.cuh"

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

// sin and cos of d pi/8, d = 0..7, in double (made on the host)
struct WindTrig {
    double s[8], c[8];
};

__global__ void k_wind_exponent(int32_t N, const float* __restrict__ ws, const float* __restrict__ wd,
                                double alpha_w1, double alpha_w2, const WindTrig T, float2* __restrict__ wexp) {
    // alpha_w1 V + alpha_w2 V (cos(d pi/4 - Theta) - 1) per env and direction, in
    // double (cos - 1 written as -2 sin^2 to avoid cancellation), split hi + lo.
    // One thread an env: sin(d pi/8 - Theta/2) = sin(d pi/8) cos(Theta/2) -
    // cos(d pi/8) sin(Theta/2), so one sincos serves the eight directions.
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N) return;
    const double V = (double)ws[e];
    double sh, ch;
    sincos(0.5 * (double)wd[e], &sh, &ch);
    float2* out = wexp + (int64_t)e * 8;
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        const double s = T.s[d] * ch - T.c[d] * sh;
        const double w = alpha_w1 * V + alpha_w2 * V * (-2.0 * s * s);
        const float hi = (float)w;
        out[d] = make_float2(hi, (float)(w - (double)hi));
    }
}

static WindTrig wind_trig() {
    WindTrig T;
    const double pi = 3.14159265358979323846;
    for (int d = 0; d < 8; ++d) {
        T.s[d] = std::sin(d * pi / 8.0);
        T.c[d] = std::cos(d * pi / 8.0);
    }
    T.c[4] = 0.0;       // cos(pi/2) exactly
    return T;
}

// wind exponent of one source cell with its own wind (per-cell mode), in double
__device__ __forceinline__ df wind_exponent_cell(float V, float Th, int d, double a1, double a2) {
    const double s = sin(0.5 * (d * 0.78539816339744830962 - (double)Th));
    const double w = a1 * (double)V + a2 * (double)V * (-2.0 * s * s);
    const float hi = (float)w;
    return {hi, (float)(w - (double)hi)};
}

__global__ void __launch_bounds__(JWF_TILE)
k_prob_table(const int2* __restrict__ tiles, int64_t n_tiles, const int32_t* __restrict__ Hs,
             const int32_t* __restrict__ Ws, const int64_t* __restrict__ offs,
             const uint8_t* __restrict__ cls, const float* __restrict__ dem,
             const float* __restrict__ ws, const float* __restrict__ wd,
             const float2* __restrict__ wexp, int per_cell_wind, const JwfDevParams P,
             const RateConsts K, float* __restrict__ q, float* __restrict__ r) {
    __shared__ RateConsts sK;
    for (int i = threadIdx.x; i < (int)(sizeof(RateConsts) / 4); i += blockDim.x)
        reinterpret_cast<float*>(&sK)[i] = reinterpret_cast<const float*>(&K)[i];
    __syncthreads();
    const double a1 = (double)P.alpha_w1, a2 = (double)P.alpha_w2;
    for (int64_t ti = blockIdx.x; ti < n_tiles; ti += gridDim.x) {
        const int2 tile = tiles[ti];
        const int e = tile.x;
        const int W = Ws[e], H = Hs[e];
        const int local = tile.y + (int)threadIdx.x;
        if (local >= H * W) continue;
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
            const float G = sK.G[cv][cls[u]];
            if (G == 0.f) continue;                      // no fuel at the source or the target
            df wx;
            if (per_cell_wind) {
                wx = wind_exponent_cell(ws[u], wd[u], d, a1, a2);
            } else {
                const float2 w2 = wexp[e * 8 + d];
                wx = {w2.x, w2.y};
            }
            rr[d] = rate_of(G, zv, dem[u], wx, d, sK);
            qq[d] = prob_of(rr[d]);
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
}

// Diagnostics of the step kernels' two-level probability (below_prob): for
// each tuple i (target and source class, elevations, wind part of the
// exponent as hi + lo, direction), out[3i .. 3i+2] = p_f, its bound B and the
// double-float probability.
__global__ void k_prob_check(int64_t n, const uint8_t* __restrict__ cv, const uint8_t* __restrict__ cu,
                             const float* __restrict__ zv, const float* __restrict__ zu,
                             const float2* __restrict__ wexp, const int32_t* __restrict__ dir, const RateConsts K,
                             float* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int d = dir[i] & 7;
        const float G = K.G[cv[i] & 15][cu[i] & 15];
        const float2 w2 = wexp[i];
        float B = 0.f;
        const float pf = prob_fast(G, zv[i], zu[i], w2.x, d, K, &B);
        out[3 * i] = pf;
        out[3 * i + 1] = B;
        out[3 * i + 2] = G == 0.f ? 0.f : prob_of(rate_of(G, zv[i], zu[i], {w2.x, w2.y}, d, K));
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

// Rate adjoint of a block of steps, on the 2-D tiles of the relaxed step:
//   gr[v][d] += sum_t glam_t(v) pb_t(v - Delta_d),  pb = (1 - m) p_burn,
// each thread summing four cells of the tile over the steps in registers (in
// step order, without branches: a zero factor adds an exact zero) and
// updating gr once, unless all its sums are zero.  Step t + 1's
// p_burn and mask (tile and a one-cell halo, zero outside the grid) and glam
// (tile) are copied to shared memory while step t is summed.
constexpr int kAccT = 256;
constexpr int kAccRows = JWF_RT_ROWS, kAccCols = JWF_RT_COLS;
constexpr int kAccW = kAccCols + 2, kAccN = (kAccRows + 2) * kAccW;
constexpr int kAccCPT = kAccRows * kAccCols / kAccT;       // cells a thread
constexpr int kAccRowStep = kAccT / kAccCols;              // rows between a thread's cells
// a step's staged planes; the mask's only when the accumulation has masks
template <bool MASKED>
struct AccStage {
    float pb[kAccN], m[kAccN];
    float gl[kAccRows * kAccCols];
};
template <>
struct AccStage<false> {
    float pb[kAccN];
    float gl[kAccRows * kAccCols];
};

// A thread's share of a step's copies, the same every step: its elements of
// the p_burn window (tile + one-cell halo) and of the glam tile, as offsets
// from the tile's first cell (halo offsets are negative; kAccOut outside the
// grid).
constexpr int kAccPbPT = (kAccN + kAccT - 1) / kAccT;          // window elements a thread
constexpr int32_t kAccOut = INT32_MIN;
struct AccPlan {
    int32_t pb[kAccPbPT];
    int32_t gl[kAccCPT];
};

__device__ __forceinline__ void acc_plan(AccPlan& pl, int y0, int x0, int H, int W) {
#pragma unroll
    for (int k = 0; k < kAccPbPT; ++k) {
        const int i = (int)threadIdx.x + k * kAccT;
        const int y = y0 - 1 + i / kAccW, x = x0 - 1 + i % kAccW;
        pl.pb[k] = (i < kAccN && y >= 0 && y < H && x >= 0 && x < W) ? (y - y0) * W + (x - x0) : kAccOut;
    }
#pragma unroll
    for (int k = 0; k < kAccCPT; ++k) {
        const int i = (int)threadIdx.x + k * kAccT;
        const int y = y0 + i / kAccCols, x = x0 + i % kAccCols;
        pl.gl[k] = (y < H && x < W) ? (y - y0) * W + (x - x0) : kAccOut;
    }
}

// copies of one step: t0 = the global index of the tile's first cell in that step's planes
template <bool MASKED>
__device__ __forceinline__ void acc_stage(AccStage<MASKED>& b, const AccPlan& pl, int64_t t0,
                                          const float* __restrict__ glam, const float* __restrict__ pburn,
                                          const float* __restrict__ mask) {
#pragma unroll
    for (int k = 0; k < kAccPbPT; ++k) {
        const int i = (int)threadIdx.x + k * kAccT;
        if (i >= kAccN) break;
        if (pl.pb[k] == kAccOut) {
            b.pb[i] = 0.f;
            if constexpr (MASKED) b.m[i] = 0.f;
            continue;
        }
        const int64_t u = t0 + pl.pb[k];
        jwf_cp_async4(&b.pb[i], pburn + u);
        if constexpr (MASKED) {
            if (mask != nullptr)
                jwf_cp_async4(&b.m[i], mask + u);
            else
                b.m[i] = 0.f;
        }
    }
#pragma unroll
    for (int k = 0; k < kAccCPT; ++k)
        if (pl.gl[k] != kAccOut) jwf_cp_async4(&b.gl[(int)threadIdx.x + k * kAccT], glam + t0 + pl.gl[k]);
}

template <bool MASKED>
__global__ void __launch_bounds__(kAccT)
k_rates_accumulate(const int4* __restrict__ tiles, const int32_t* __restrict__ Hs, const int32_t* __restrict__ Ws,
                   const int64_t* __restrict__ offs, int64_t cells, int32_t n_steps,
                   const float* __restrict__ glam, const float* __restrict__ pburn,
                   const float* __restrict__ mask, float* __restrict__ gr) {
    __shared__ __align__(16) AccStage<MASKED> st[2];
    const int4 tl = tiles[blockIdx.x];
    const int e = tl.x, y0 = tl.y, x0 = tl.z;
    const int H = Hs[e], W = Ws[e];
    const int64_t off = offs[e];
    const int tx = (int)threadIdx.x % kAccCols, ty = (int)threadIdx.x / kAccCols;
    float w[kAccCPT][8];
#pragma unroll
    for (int k = 0; k < kAccCPT; ++k)
#pragma unroll
        for (int d = 0; d < 8; ++d) w[k][d] = 0.f;
    AccPlan pl;
    acc_plan(pl, y0, x0, H, W);
    const int64_t tile0 = off + (int64_t)y0 * W + x0;
    acc_stage(st[0], pl, tile0, glam, pburn, mask);
    jwf_cp_async_commit();
    for (int t = 0; t < n_steps; ++t) {
        if (t + 1 < n_steps)
            acc_stage(st[(t + 1) & 1], pl, (int64_t)(t + 1) * cells + tile0, glam, pburn, mask);
        jwf_cp_async_commit();
        jwf_cp_async_wait_prev();
        __syncthreads();
        AccStage<MASKED>& b = st[t & 1];
#pragma unroll
        for (int k = 0; k < kAccCPT; ++k) {
            const int ly = ty + k * kAccRowStep;
            if (y0 + ly >= H || x0 + tx >= W) continue;
            const float g = b.gl[ly * kAccCols + tx];
#pragma unroll
            for (int d = 0; d < 8; ++d) {
                const int li = (ly + 1 - jwf_dr(d)) * kAccW + (tx + 1 - jwf_dx(d));
                float pb = b.pb[li];
                if constexpr (MASKED) {
                    if (mask != nullptr) pb *= 1.0f - b.m[li];
                }
                w[k][d] += g * pb;
            }
        }
        __syncthreads();
    }
    bool any = false;
#pragma unroll
    for (int k = 0; k < kAccCPT; ++k)
#pragma unroll
        for (int d = 0; d < 8; ++d) any = any || w[k][d] != 0.f;
    if (!any) return;
#pragma unroll
    for (int k = 0; k < kAccCPT; ++k) {
        const int y = y0 + ty + k * kAccRowStep, x = x0 + tx;
        if (y >= H || x >= W) continue;
        float4* g4 = reinterpret_cast<float4*>(gr + (off + (int64_t)y * W + x) * 8);
        float4 a = g4[0], c = g4[1];
        a.x += w[k][0]; a.y += w[k][1]; a.z += w[k][2]; a.w += w[k][3];
        c.x += w[k][4]; c.y += w[k][5]; c.z += w[k][6]; c.w += w[k][7];
        g4[0] = a;
        g4[1] = c;
    }
}

// Parameter gradient through the rates.  Per target cell v and direction d
// (source u = v - Delta_d), w = gr[v][d] is the adjoint of r(v, d); with
// r = gamma(v) phi(u, d),
//   dr/dp_base = gamma A_u K,   dr/dalpha_gamma = A_v phi,
//   dr/dalpha_w1 = r V,  dr/dalpha_w2 = r V (cos - 1),  dr/dalpha_s = r S,
//   dr/dmu_veg[k] = (1 + mu_den[k]) B_k,  dr/dmu_den[k] = (1 + mu_veg[k]) B_k,
// where B_k gathers alpha_gamma phi (target of class k) and gamma p_base K
// (source of class k); no division, so classes without fuel are exact.
// Each thread sums its cells in float (a few dozen terms); the class bins sit
// in shared memory, one column per thread (class-major, conflict-free); the
// block and the grid are reduced in double in a fixed order (the last block
// to finish adds the per-block partials), so the result is deterministic.
template <int C>
__global__ void __launch_bounds__(kRbThreads)
k_rates_bwd(const int2* __restrict__ tiles, int64_t n_tiles, const int32_t* __restrict__ Hs,
            const int32_t* __restrict__ Ws, const int64_t* __restrict__ offs, int64_t cells,
            const float* __restrict__ gr, const uint8_t* __restrict__ cls,
            const float* __restrict__ dem, const float* __restrict__ ws,
            const float* __restrict__ wd, int per_cell_wind, const JwfDevParams P,
            double* __restrict__ partials, uint32_t* __restrict__ counter,
            double* __restrict__ gparams) {
    constexpr int NV = kRbScalars + 2 * C;
    __shared__ float bins[C * kRbThreads];
    __shared__ double red[kRbThreads];
    __shared__ bool am_last;
    const int tid = threadIdx.x;
    for (int k = 0; k < C; ++k) bins[k * kRbThreads + tid] = 0.f;
    float g_pb = 0.f, g_w1 = 0.f, g_w2 = 0.f, g_s = 0.f, g_gam = 0.f;
    const DirConst dc = dir_const();
    const float slope_scale = 57.295779513082320876f;
    const float inv_cell = 1.0f / P.cell_size;

    for (int64_t ti = blockIdx.x; ti < n_tiles; ti += gridDim.x) {
        const int2 tile = tiles[ti];
        const int e = tile.x;
        const int W = Ws[e], H = Hs[e];
        const int local = tile.y + tid;
        if (local >= H * W) continue;
        const int64_t off = offs[e];
        const int y = local / W, x = local - (local / W) * W;
        const int64_t v = off + local;
        const float4* g4 = reinterpret_cast<const float4*>(gr + v * 8);
        const float4 ga = __ldg(g4), gb = __ldg(g4 + 1);
        const float w[8] = {ga.x, ga.y, ga.z, ga.w, gb.x, gb.y, gb.z, gb.w};
        const int cv = cls[v];
        const float zv = dem[v];
        const float Av = (1.0f + P.mu_veg[cv]) * (1.0f + P.mu_den[cv]);
        const float gamma = P.alpha_gamma * Av;
        float cth = 0.f, sth = 0.f, Venv = 0.f;
        if (!per_cell_wind) {
            Venv = ws[e];
            sincosf(wd[e], &sth, &cth);
        }
        float tgt = 0.f;
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            if (w[d] == 0.f) continue;
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
            const float wr = w[d] * gamma * phi;
            g_pb += w[d] * gamma * Au * t.K;
            g_w1 += wr * t.V;
            g_w2 += wr * t.V * t.cosm1;
            g_s += wr * t.S;
            g_gam += w[d] * Av * phi;
            tgt += w[d] * phi;
            bins[cu * kRbThreads + tid] += w[d] * gamma * P.p_base * t.K;   // source of class cu
        }
        if (tgt != 0.f) bins[cv * kRbThreads + tid] += P.alpha_gamma * tgt;  // target of class cv
    }
    // block reduction in double, fixed order: thread values -> red[] tree
    const float sc[kRbScalars] = {g_pb, g_w1, g_w2, g_s, g_gam};
#pragma unroll 1
    for (int i = 0; i < NV; ++i) {
        double val;
        if (i < kRbScalars) {
            val = (double)(i == 0 ? sc[0] : i == 1 ? sc[1] : i == 2 ? sc[2] : i == 3 ? sc[3] : sc[4]);
        } else {
            const int k = (i - kRbScalars) % C;
            const float b = bins[k * kRbThreads + tid];
            val = (i - kRbScalars) < C ? (double)(b * (1.0f + P.mu_den[k])) : (double)(b * (1.0f + P.mu_veg[k]));
        }
        red[tid] = val;
        __syncthreads();
        for (int o = kRbThreads / 2; o > 0; o >>= 1) {
            if (tid < o) red[tid] += red[tid + o];
            __syncthreads();
        }
        if (tid == 0) partials[(int64_t)blockIdx.x * NV + i] = red[0];
        __syncthreads();
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) am_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    // the last block sums the block partials in a fixed order
    const int nC = P.n_classes;
#pragma unroll 1
    for (int i = 0; i < NV; ++i) {
        double s2 = 0.0;
        for (int b = tid; b < (int)gridDim.x; b += kRbThreads) s2 += __ldcg(&partials[(int64_t)b * NV + i]);
        red[tid] = s2;
        __syncthreads();
        for (int o = kRbThreads / 2; o > 0; o >>= 1) {
            if (tid < o) red[tid] += red[tid + o];
            __syncthreads();
        }
        if (tid == 0) {
            // layout [p_base, alpha_w1, alpha_w2, alpha_s, alpha_gamma, mu_veg[nC], mu_den[nC]]
            const double g = red[0];
            if (i < kRbScalars) {
                gparams[i] += g;
            } else if (i < kRbScalars + C) {
                if (i - kRbScalars < nC) gparams[i] += g;
            } else {
                const int k = i - kRbScalars - C;
                if (k < nC) gparams[kRbScalars + nC + k] += g;
            }
        }
        __syncthreads();
    }
    if (tid == 0) *counter = 0u;
}

template <int C>
cudaError_t launch_rates_contract_c(jwf_ctx* c, const float* gr, const uint8_t* cls, const float* dem,
                                    const float* ws, const float* wd, double* gparams, cudaStream_t s) {
    constexpr int NV = kRbScalars + 2 * C;
    int64_t grid = (int64_t)c->num_sms * 6;
    if (grid > c->n_tiles) grid = c->n_tiles;
    if (grid * NV > c->partial_cap) grid = c->partial_cap / NV;
    if (grid < 1) return cudaErrorInvalidValue;
    k_rates_bwd<C><<<(unsigned)grid, kRbThreads, 0, s>>>(
        c->d_tiles, c->n_tiles, c->d_H, c->d_W, c->d_off, c->cells, gr, cls, dem, ws, wd,
        (c->flags & JWF_WIND_PER_CELL) ? 1 : 0, c->P, c->d_partials, c->d_red_counter, gparams);
    return cudaGetLastError();
}

}  // namespace

static df split_df(double v) {
    const float hi = (float)v;
    return {hi, (float)(v - (double)hi)};
}

void jwf_rate_consts(const jwf_ctx* c, RateConsts* K) {
    const double pi = 3.14159265358979323846;
    *K = RateConsts{};
    for (int k = 0; k <= 64; ++k) {
        const double th = k * pi / 256.0;
        K->atan_th[k] = split_df(th);
        K->atan_tan[k] = split_df(std::tan(th));
    }
    K->half_pi = split_df(pi / 2.0);
    K->slope_coef = split_df((double)c->P.alpha_s * 180.0 / pi);
    for (int d = 0; d < 8; ++d)
        K->inv_run[d] = split_df(1.0 / ((double)c->P.cell_size * ((d & 1) ? std::sqrt(2.0) : 1.0)));
    for (int a = 0; a < 16; ++a)
        for (int b = 0; b < 16; ++b) {
            if (a >= c->n_classes || b >= c->n_classes) {
                K->G[a][b] = 0.f;
                continue;
            }
            const double gamma = (double)c->P.alpha_gamma * (1.0 + (double)c->P.mu_veg[a]) *
                                 (1.0 + (double)c->P.mu_den[a]);
            const double base = (double)c->P.p_base * (1.0 + (double)c->P.mu_veg[b]) *
                                (1.0 + (double)c->P.mu_den[b]);
            K->G[a][b] = (float)(gamma * base);
        }
}

cudaError_t jwf_launch_prob_check(const jwf_ctx* c, int64_t n, const uint8_t* cv, const uint8_t* cu,
                                  const float* zv, const float* zu, const float* wexp, const int32_t* dir,
                                  float* out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    RateConsts K;
    jwf_rate_consts(c, &K);
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, (int64_t)c->num_sms * 8);
    k_prob_check<<<(unsigned)blocks, 256, 0, s>>>(n, cv, cu, zv, zu, reinterpret_cast<const float2*>(wexp), dir, K,
                                                   out);
    return cudaGetLastError();
}

cudaError_t jwf_launch_wind_exponent(const jwf_ctx* c, const float* ws, const float* wd, cudaStream_t s) {
    k_wind_exponent<<<(c->N + 127) / 128, 128, 0, s>>>(c->N, ws, wd, (double)c->P.alpha_w1,
                                                         (double)c->P.alpha_w2, wind_trig(), c->d_wexp);
    return cudaGetLastError();
}

cudaError_t jwf_launch_wind_series(jwf_ctx* c, cudaStream_t s) {
    // the series is [steps][N]: the same kernel over steps x N "envs"
    const int64_t n = (int64_t)c->wser_n * c->N;
    if (n == 0) return cudaSuccess;
    k_wind_exponent<<<(unsigned)((n + 127) / 128), 128, 0, s>>>((int32_t)n, c->s_ws, c->s_wd,
                                                               (double)c->P.alpha_w1, (double)c->P.alpha_w2,
                                                               wind_trig(), c->d_wser);
    return cudaGetLastError();
}

cudaError_t jwf_launch_prob_table(const jwf_ctx* c, const uint8_t* cls, const float* dem,
                                  const float* ws, const float* wd, cudaStream_t s) {
    RateConsts K;
    jwf_rate_consts(c, &K);
    const bool per_cell = (c->flags & JWF_WIND_PER_CELL) != 0u;
    if (!per_cell) {
        const cudaError_t err = jwf_launch_wind_exponent(c, ws, wd, s);
        if (err != cudaSuccess) return err;
    }
    int64_t grid = (int64_t)c->num_sms * 8;
    if (grid > c->n_tiles) grid = c->n_tiles;
    k_prob_table<<<(unsigned)grid, JWF_TILE, 0, s>>>(
        c->d_tiles, c->n_tiles, c->d_H, c->d_W, c->d_off, cls, dem, ws, wd, c->d_wexp, per_cell ? 1 : 0,
        c->P, K, c->d_q, (c->flags & JWF_KEEP_RATES) ? c->d_r : nullptr);
    return cudaGetLastError();
}

cudaError_t jwf_launch_rates_accumulate(const jwf_ctx* c, int32_t n_steps, const float* glam,
                                        const float* pburn, const float* mask, float* gr, cudaStream_t s) {
    if (mask != nullptr)
        k_rates_accumulate<true><<<(unsigned)c->n_rtiles, kAccT, 0, s>>>(c->d_rtiles, c->d_H, c->d_W, c->d_off,
                                                                      c->cells, n_steps, glam, pburn, mask, gr);
    else
        k_rates_accumulate<false><<<(unsigned)c->n_rtiles, kAccT, 0, s>>>(c->d_rtiles, c->d_H, c->d_W, c->d_off,
                                                                       c->cells, n_steps, glam, pburn, mask, gr);
    return cudaGetLastError();
}

cudaError_t jwf_launch_rates_contract(jwf_ctx* c, const float* gr, const uint8_t* cls, const float* dem,
                                      const float* ws, const float* wd, double* gparams, cudaStream_t s) {
    // class-count specialisations keep the per-class bins sized to the table
    const int C = c->n_classes;
    if (C <= 1) return launch_rates_contract_c<1>(c, gr, cls, dem, ws, wd, gparams, s);
    if (C <= 4) return launch_rates_contract_c<4>(c, gr, cls, dem, ws, wd, gparams, s);
    if (C <= 11) return launch_rates_contract_c<11>(c, gr, cls, dem, ws, wd, gparams, s);
    if (C <= 16) return launch_rates_contract_c<16>(c, gr, cls, dem, ws, wd, gparams, s);
    return cudaErrorNotSupported;
}

cudaError_t jwf_launch_rates_bwd(jwf_ctx* c, int32_t n_steps, const float* glam,
                                 const float* pburn, const float* mask, const uint8_t* cls,
                                 const float* dem, const float* ws, const float* wd,
                                 double* gparams, cudaStream_t s) {
    cudaError_t err = cudaMemsetAsync(c->d_gr, 0, (size_t)c->cells * 8 * sizeof(float), s);
    if (err == cudaSuccess) err = jwf_launch_rates_accumulate(c, n_steps, glam, pburn, mask, c->d_gr, s);
    if (err == cudaSuccess) err = jwf_launch_rates_contract(c, c->d_gr, cls, dem, ws, wd, gparams, s);
    return err;
}
