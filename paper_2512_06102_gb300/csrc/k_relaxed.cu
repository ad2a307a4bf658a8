// k_relaxed.cu -- deterministic (raw-probabilities) update, Section 3,
// Eqs. 5-10, with p_ignite from Eq. 4 (b(u) replaced by p_burn(u)), and its
// adjoint.
//
// Forward, per cell v (pb = (1 - m) p_burn: the tanker acts first):
//   lam = sum_d pb(v - Delta_d) r[v][d];  p_ign = 1 - exp(-lam)
//   p_un' = p_un - p_un p_ign;  p_burn' = p_un p_ign + p_continue pb(v)
// Adjoint, given a_u = dL/dp_un', a_b = dL/dp_burn':
//   nb    = a_b - a_u
//   dL/dp_un(v)  = a_u + nb p_ign
//   glam(v)      = nb p_un exp(-lam)                    (= dL/dlam(v))
//   dL/dp_burn(u) = (1 - m(u)) (p_continue a_b(u) + sum_d glam(u + Delta_d) r[u + Delta_d][d])
//   dL/dp_continue = sum_v a_b(v) pb(v)
// HBM-bound stencils: the forward moves 8 B of state in, 32 B of rates and
// 8 B of state out per cell.  The plain kernels split the adjoint in two
// passes (glam, then the transpose gather) so that no cell recomputes a
// neighbour's lam; the tiled set does it in one column sweep.
//
// The adjoint of a cell that the fire has not reached grows by about
// sum_d r per step (a spark there would spread), so it can leave the float
// range over long horizons.  Every stored adjoint is therefore saturated at
// +-JWF_ADJ_SAT (1e35): with rates below ~3e36 / 9 no sum of nine terms can
// overflow, so the adjoint never becomes inf or NaN.  Only entries whose
// exact value exceeds 1e35 are affected (they lie ahead of the fire, where
// p_burn is zero, so the parameter gradients do not see them); a factor that
// is exactly zero keeps its product zero.
#include "jwf_internal.cuh"

namespace {

constexpr float JWF_ADJ_SAT = 1e35f;

__device__ __forceinline__ float sat(float x) { return fminf(fmaxf(x, -JWF_ADJ_SAT), JWF_ADJ_SAT); }

__device__ __forceinline__ float pb_at(const float* __restrict__ pburn, const float* __restrict__ mask,
                                       int64_t i) {
    const float p = pburn[i];
    return mask != nullptr ? p * (1.0f - mask[i]) : p;
}

__global__ void __launch_bounds__(JWF_TILE)
k_relaxed_fwd(const int2* __restrict__ tiles, const int32_t* __restrict__ Hs,
              const int32_t* __restrict__ Ws, const int64_t* __restrict__ offs,
              const float* __restrict__ r, const float* __restrict__ pun,
              const float* __restrict__ pburn, const float* __restrict__ mask, float p_continue,
              float* __restrict__ pun_out, float* __restrict__ pburn_out) {
    const int2 tile = tiles[blockIdx.x];
    const int e = tile.x;
    const int W = Ws[e], H = Hs[e];
    const int local = tile.y + (int)threadIdx.x;
    if (local >= H * W) return;
    const int64_t off = offs[e];
    const int y = local / W, x = local - (local / W) * W;
    const int64_t v = off + local;
    const float4* r4 = reinterpret_cast<const float4*>(r + v * 8);
    const float4 ra = __ldg(r4), rb = __ldg(r4 + 1);
    const float rv[8] = {ra.x, ra.y, ra.z, ra.w, rb.x, rb.y, rb.z, rb.w};
    float lam = 0.f;
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        const int uy = y - jwf_dr(d), ux = x - jwf_dx(d);
        if (uy < 0 || uy >= H || ux < 0 || ux >= W) continue;
        lam += pb_at(pburn, mask, off + (int64_t)uy * W + ux) * rv[d];
    }
    const float p_ign = -expm1f(-lam);
    const float pu = pun[v];
    const float newly = pu * p_ign;
    pun_out[v] = pu - newly;
    pburn_out[v] = newly + p_continue * pb_at(pburn, mask, v);
}

// pass A: dL/dp_un, glam, and the p_continue partial sums
__global__ void __launch_bounds__(JWF_TILE)
k_relaxed_bwd_a(const int2* __restrict__ tiles, int64_t n_tiles, const int32_t* __restrict__ Hs,
                const int32_t* __restrict__ Ws, const int64_t* __restrict__ offs,
                const float* __restrict__ r, const float* __restrict__ pun,
                const float* __restrict__ pburn, const float* __restrict__ mask,
                const float* __restrict__ gun_out, const float* __restrict__ gburn_out,
                float* __restrict__ gun, float* __restrict__ glam, double* __restrict__ partials,
                uint32_t* __restrict__ counter, double* __restrict__ gpc) {
    __shared__ double red[JWF_TILE / 32];
    __shared__ bool am_last;
    double acc = 0.0;
    for (int64_t ti = blockIdx.x; ti < n_tiles; ti += gridDim.x) {
        const int2 tile = tiles[ti];
        const int e = tile.x;
        const int W = Ws[e], H = Hs[e];
        const int local = tile.y + (int)threadIdx.x;
        if (local >= H * W) continue;
        const int64_t off = offs[e];
        const int y = local / W, x = local - (local / W) * W;
        const int64_t v = off + local;
        const float4* r4 = reinterpret_cast<const float4*>(r + v * 8);
        const float4 ra = __ldg(r4), rb = __ldg(r4 + 1);
        const float rv[8] = {ra.x, ra.y, ra.z, ra.w, rb.x, rb.y, rb.z, rb.w};
        float lam = 0.f;
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            const int uy = y - jwf_dr(d), ux = x - jwf_dx(d);
            if (uy < 0 || uy >= H || ux < 0 || ux >= W) continue;
            lam += pb_at(pburn, mask, off + (int64_t)uy * W + ux) * rv[d];
        }
        const float em = expf(-lam);
        const float p_ign = -expm1f(-lam);
        const float au = gun_out[v], ab = gburn_out[v];
        const float nb = ab - au;
        const float pe = pun[v] * em;
        gun[v] = sat(p_ign != 0.f ? au + nb * p_ign : au);
        glam[v] = pe != 0.f ? sat(nb * pe) : 0.f;
        const float pbv = pb_at(pburn, mask, v);
        if (pbv != 0.f) acc += (double)(ab * pbv);
    }
    // deterministic reduction of the p_continue gradient
    if (gpc == nullptr) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < JWF_TILE / 32; ++w) s += red[w];
        partials[blockIdx.x] = s;
        __threadfence();
        am_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    double s = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) s += __ldcg(&partials[b]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < JWF_TILE / 32; ++w) tot += red[w];
        *gpc += tot;
        *counter = 0u;
    }
}

// pass B: dL/dp_burn(u) gathers glam of the targets u feeds
__global__ void __launch_bounds__(JWF_TILE)
k_relaxed_bwd_b(const int2* __restrict__ tiles, const int32_t* __restrict__ Hs,
                const int32_t* __restrict__ Ws, const int64_t* __restrict__ offs,
                const float* __restrict__ r, const float* __restrict__ mask,
                const float* __restrict__ gburn_out, const float* __restrict__ glam,
                float p_continue, float* __restrict__ gburn) {
    const int2 tile = tiles[blockIdx.x];
    const int e = tile.x;
    const int W = Ws[e], H = Hs[e];
    const int local = tile.y + (int)threadIdx.x;
    if (local >= H * W) return;
    const int64_t off = offs[e];
    const int y = local / W, x = local - (local / W) * W;
    const int64_t u = off + local;
    float g = p_continue != 0.f ? p_continue * gburn_out[u] : 0.f;
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        const int vy = y + jwf_dr(d), vx = x + jwf_dx(d);   // target v = u + Delta_d
        if (vy < 0 || vy >= H || vx < 0 || vx >= W) continue;
        const int64_t v = off + (int64_t)vy * W + vx;
        const float rv = __ldg(r + v * 8 + d);
        const float gl = glam[v];
        if (rv != 0.f && gl != 0.f) g += gl * rv;
    }
    if (mask != nullptr) {
        const float keep = 1.0f - mask[u];
        g = keep != 0.f ? g * keep : 0.f;
    }
    gburn[u] = sat(g);
}

// ---------------------------------------------------------------------------
// Tiled variant: the forward walks 2-D tiles of kRH x kRW cells staged in
// shared memory by asynchronous copies; each warp covers 32 consecutive cells
// of a row, so the rate rows (32 B a cell) stream in 1 KB runs.  The adjoint
// is a column sweep (below): one kernel, no glam round trip, each rate row
// read once.
constexpr int kRH = JWF_RT_ROWS, kRW = JWF_RT_COLS;


// Forward: two persistent CTAs per SM walk the tiles, two tiles deep: the
// copies of the next tile (rate rows and p_un of the tile, p_burn and the
// mask of the tile and a one-cell halo, zero outside the grid) are in flight
// while the current one is computed.
constexpr int kFT = 256;                                   // threads of the forward CTA
constexpr int kFW = kRW + 2, kFN = (kRH + 2) * kFW;        // tile + 1: pb
struct FwdStage {
    float r[kRH * kRW * 8];
    float pu[kRH * kRW];
    float pb[kFN], m[kFN];
};
struct FwdSmem {
    FwdStage st[2];
};
size_t fwd_smem_bytes() { return sizeof(FwdSmem); }

__device__ __forceinline__ void fwd_stage(FwdStage& b, const int4* __restrict__ tiles, int64_t ti,
                                          const int32_t* __restrict__ Hs, const int32_t* __restrict__ Ws,
                                          const int64_t* __restrict__ offs, const float* __restrict__ r,
                                          const float* __restrict__ pun, const float* __restrict__ pburn,
                                          const float* __restrict__ mask) {
    const int4 tl = tiles[ti];
    const int e = tl.x, y0 = tl.y, x0 = tl.z;
    const int H = Hs[e], W = Ws[e];
    const int64_t off = offs[e];
    for (int i = threadIdx.x; i < kRH * kRW; i += kFT) {
        const int y = y0 + i / kRW, x = x0 + i % kRW;
        if (y >= H || x >= W) continue;
        const int64_t v = off + (int64_t)y * W + x;
        jwf_cp_async16(&b.r[i * 8], r + v * 8);
        jwf_cp_async16(&b.r[i * 8 + 4], r + v * 8 + 4);
        jwf_cp_async4(&b.pu[i], pun + v);
    }
    for (int i = threadIdx.x; i < kFN; i += kFT) {
        const int y = y0 - 1 + i / kFW, x = x0 - 1 + i % kFW;
        if (y < 0 || y >= H || x < 0 || x >= W) {
            b.pb[i] = 0.f;
            b.m[i] = 0.f;
            continue;
        }
        const int64_t v = off + (int64_t)y * W + x;
        jwf_cp_async4(&b.pb[i], pburn + v);
        if (mask != nullptr)
            jwf_cp_async4(&b.m[i], mask + v);
        else
            b.m[i] = 0.f;
    }
}

__global__ void __launch_bounds__(kFT)
k_relaxed_fwd_tiled(const int4* __restrict__ tiles, int64_t n_tiles, const int32_t* __restrict__ Hs,
                    const int32_t* __restrict__ Ws, const int64_t* __restrict__ offs,
                    const float* __restrict__ r, const float* __restrict__ pun,
                    const float* __restrict__ pburn, const float* __restrict__ mask, float p_continue,
                    float* __restrict__ pun_out, float* __restrict__ pburn_out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FwdSmem& S = *reinterpret_cast<FwdSmem*>(smem_raw);
    int cur = 0;
    if ((int64_t)blockIdx.x < n_tiles) fwd_stage(S.st[0], tiles, blockIdx.x, Hs, Ws, offs, r, pun, pburn, mask);
    jwf_cp_async_commit();
    for (int64_t ti = blockIdx.x; ti < n_tiles; ti += gridDim.x, cur ^= 1) {
        if (ti + gridDim.x < n_tiles)
            fwd_stage(S.st[cur ^ 1], tiles, ti + gridDim.x, Hs, Ws, offs, r, pun, pburn, mask);
        jwf_cp_async_commit();
        const int4 tl = tiles[ti];
        const int e = tl.x, y0 = tl.y, x0 = tl.z;
        const int H = Hs[e], W = Ws[e];
        const int64_t off = offs[e];
        jwf_cp_async_wait_prev();
        __syncthreads();
        FwdStage& b = S.st[cur];
        if (mask != nullptr) {
            for (int i = threadIdx.x; i < kFN; i += kFT) b.pb[i] = b.pb[i] * (1.0f - b.m[i]);
            __syncthreads();
        }
        for (int j = threadIdx.x; j < kRH * kRW; j += kFT) {
            const int ty = j / kRW, tx = j - (j / kRW) * kRW;
            const int y = y0 + ty, x = x0 + tx;
            if (y >= H || x >= W) continue;
            const float4 ra = *reinterpret_cast<const float4*>(&b.r[j * 8]);
            const float4 rb = *reinterpret_cast<const float4*>(&b.r[j * 8 + 4]);
            const float rv[8] = {ra.x, ra.y, ra.z, ra.w, rb.x, rb.y, rb.z, rb.w};
            float lam = 0.f;
#pragma unroll
            for (int d = 0; d < 8; ++d) lam += b.pb[(ty + 1 - jwf_dr(d)) * kFW + (tx + 1 - jwf_dx(d))] * rv[d];
            const float p_ign = -expm1f(-lam);
            const float pu = b.pu[j];
            const float newly = pu * p_ign;
            const int64_t v = off + (int64_t)y * W + x;
            pun_out[v] = pu - newly;
            pburn_out[v] = newly + p_continue * b.pb[(ty + 1) * kFW + tx + 1];
        }
        __syncthreads();
    }
}

// Two steps per pass.  A tile of kR2H x kR2W output cells is staged with a
// two-cell halo: step t runs on the tile and the ring of cells around it
// (whose burning probabilities step t + 1 reads), step t + 1 on the tile, so
// each rate row is read once for both steps (32 B a cell plus the halo's
// share, instead of 2 x 32 B).  Both steps write the tile's states; every
// cell's arithmetic is the one-step kernel's, so the results are identical.
constexpr int kR2H = JWF_R2_ROWS, kR2W = JWF_R2_COLS;
constexpr int kF2T = 256;                                           // threads of the two-step CTA
constexpr int kA1H = kR2H + 2, kA1W = kR2W + 2, kA1N = kA1H * kA1W;  // cells of step t (tile + 1)
constexpr int kA0H = kR2H + 4, kA0W = kR2W + 4, kA0N = kA0H * kA0W;  // p_burn read by step t (tile + 2)
// A stage's buffers; the masks' only when the pass has tanker masks (without
// them a CTA needs less shared memory and more CTAs fit an SM).
template <bool MASKED>
struct Fwd2Stage {
    float r[kA1N * 8];
    float pu[kA1N];
    float pb[kA0N], m0[kA0N];
    float m1[kA1N];
};
template <>
struct Fwd2Stage<false> {
    float r[kA1N * 8];
    float pu[kA1N];
    float pb[kA0N];
};
template <bool MASKED>
struct Fwd2Smem {
    Fwd2Stage<MASKED> st[2];
    float pb1[kA1N];    // p_burn after step t (masked for step t + 1 before use)
    float pu1[kA1N];    // p_un after step t
};
template <bool MASKED>
size_t fwd2_smem_bytes() {
    return sizeof(Fwd2Smem<MASKED>);
}

template <bool MASKED>
__device__ __forceinline__ void fwd2_stage(Fwd2Stage<MASKED>& b, const int4* __restrict__ tiles, int64_t ti,
                                           const int32_t* __restrict__ Hs, const int32_t* __restrict__ Ws,
                                           const int64_t* __restrict__ offs, const float* __restrict__ r,
                                           const float* __restrict__ pun, const float* __restrict__ pburn,
                                           const float* __restrict__ mask0, const float* __restrict__ mask1) {
    const int4 tl = tiles[ti];
    const int e = tl.x, y0 = tl.y, x0 = tl.z;
    const int H = Hs[e], W = Ws[e];
    const int64_t off = offs[e];
    for (int i = threadIdx.x; i < kA1N; i += kF2T) {
        const int y = y0 - 1 + i / kA1W, x = x0 - 1 + i % kA1W;
        if (y < 0 || y >= H || x < 0 || x >= W) {
            b.pu[i] = 0.f;
            if constexpr (MASKED) b.m1[i] = 0.f;
            continue;
        }
        const int64_t v = off + (int64_t)y * W + x;
        jwf_cp_async16(&b.r[i * 8], r + v * 8);
        jwf_cp_async16(&b.r[i * 8 + 4], r + v * 8 + 4);
        jwf_cp_async4(&b.pu[i], pun + v);
        if constexpr (MASKED) {
            if (mask1 != nullptr)
                jwf_cp_async4(&b.m1[i], mask1 + v);
            else
                b.m1[i] = 0.f;
        }
    }
    for (int i = threadIdx.x; i < kA0N; i += kF2T) {
        const int y = y0 - 2 + i / kA0W, x = x0 - 2 + i % kA0W;
        if (y < 0 || y >= H || x < 0 || x >= W) {
            b.pb[i] = 0.f;
            if constexpr (MASKED) b.m0[i] = 0.f;
            continue;
        }
        const int64_t v = off + (int64_t)y * W + x;
        jwf_cp_async4(&b.pb[i], pburn + v);
        if constexpr (MASKED) {
            if (mask0 != nullptr)
                jwf_cp_async4(&b.m0[i], mask0 + v);
            else
                b.m0[i] = 0.f;
        }
    }
}

template <bool MASKED>
__global__ void __launch_bounds__(kF2T)
k_relaxed_fwd2_tiled(const int4* __restrict__ tiles, int64_t n_tiles, const int32_t* __restrict__ Hs,
                     const int32_t* __restrict__ Ws, const int64_t* __restrict__ offs,
                     const float* __restrict__ r, const float* __restrict__ pun,
                     const float* __restrict__ pburn, const float* __restrict__ mask0,
                     const float* __restrict__ mask1, float p_continue, float* __restrict__ pun1,
                     float* __restrict__ pburn1, float* __restrict__ pun2, float* __restrict__ pburn2) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Fwd2Smem<MASKED>& S = *reinterpret_cast<Fwd2Smem<MASKED>*>(smem_raw);
    int cur = 0;
    if ((int64_t)blockIdx.x < n_tiles)
        fwd2_stage(S.st[0], tiles, blockIdx.x, Hs, Ws, offs, r, pun, pburn, mask0, mask1);
    jwf_cp_async_commit();
    for (int64_t ti = blockIdx.x; ti < n_tiles; ti += gridDim.x, cur ^= 1) {
        if (ti + gridDim.x < n_tiles)
            fwd2_stage(S.st[cur ^ 1], tiles, ti + gridDim.x, Hs, Ws, offs, r, pun, pburn, mask0, mask1);
        jwf_cp_async_commit();
        const int4 tl = tiles[ti];
        const int e = tl.x, y0 = tl.y, x0 = tl.z;
        const int H = Hs[e], W = Ws[e];
        const int64_t off = offs[e];
        jwf_cp_async_wait_prev();
        __syncthreads();
        Fwd2Stage<MASKED>& b = S.st[cur];
        if constexpr (MASKED) {
            if (mask0 != nullptr) {
                for (int q = threadIdx.x; q < kA0N; q += kF2T) b.pb[q] = b.pb[q] * (1.0f - b.m0[q]);
                __syncthreads();
            }
        }
        // step t on the tile and its one-cell ring
        for (int j = threadIdx.x; j < kA1N; j += kF2T) {
            const int ay = j / kA1W, ax = j - (j / kA1W) * kA1W;
            const int y = y0 - 1 + ay, x = x0 - 1 + ax;
            if (y < 0 || y >= H || x < 0 || x >= W) {
                S.pb1[j] = 0.f;
                S.pu1[j] = 0.f;
                continue;
            }
            const float4 ra = *reinterpret_cast<const float4*>(&b.r[j * 8]);
            const float4 rb = *reinterpret_cast<const float4*>(&b.r[j * 8 + 4]);
            const float rv[8] = {ra.x, ra.y, ra.z, ra.w, rb.x, rb.y, rb.z, rb.w};
            float lam = 0.f;
#pragma unroll
            for (int d = 0; d < 8; ++d) lam += b.pb[(ay + 1 - jwf_dr(d)) * kA0W + (ax + 1 - jwf_dx(d))] * rv[d];
            const float p_ign = -expm1f(-lam);
            const float pu = b.pu[j];
            const float newly = pu * p_ign;
            const float u1 = pu - newly;
            const float b1 = newly + p_continue * b.pb[(ay + 1) * kA0W + ax + 1];
            S.pu1[j] = u1;
            S.pb1[j] = b1;
            if (ay >= 1 && ay <= kR2H && ax >= 1 && ax <= kR2W) {
                const int64_t v = off + (int64_t)y * W + x;
                pun1[v] = u1;
                pburn1[v] = b1;
            }
        }
        __syncthreads();
        if constexpr (MASKED) {
            if (mask1 != nullptr) {
                for (int q = threadIdx.x; q < kA1N; q += kF2T) S.pb1[q] = S.pb1[q] * (1.0f - b.m1[q]);
                __syncthreads();
            }
        }
        // step t + 1 on the tile
        for (int j = threadIdx.x; j < kR2H * kR2W; j += kF2T) {
            const int ty = j / kR2W, tx = j - (j / kR2W) * kR2W;
            const int y = y0 + ty, x = x0 + tx;
            if (y >= H || x >= W) continue;
            const int a1 = (ty + 1) * kA1W + (tx + 1);
            const float4 ra = *reinterpret_cast<const float4*>(&b.r[a1 * 8]);
            const float4 rb = *reinterpret_cast<const float4*>(&b.r[a1 * 8 + 4]);
            const float rv[8] = {ra.x, ra.y, ra.z, ra.w, rb.x, rb.y, rb.z, rb.w};
            float lam = 0.f;
#pragma unroll
            for (int d = 0; d < 8; ++d) lam += S.pb1[(ty + 1 - jwf_dr(d)) * kA1W + (tx + 1 - jwf_dx(d))] * rv[d];
            const float p_ign = -expm1f(-lam);
            const float pu = S.pu1[a1];
            const float newly = pu * p_ign;
            const int64_t v = off + (int64_t)y * W + x;
            pun2[v] = pu - newly;
            pburn2[v] = newly + p_continue * S.pb1[a1];
        }
        __syncthreads();
    }
}

// Column-sweep adjoint.  A warp owns a strip of JWF_SW_COLS output columns
// (lane L is column x0 - 1 + L: lanes 0 and 31 are halo columns) and walks
// down rows y0 - 1 .. y1, one target row per iteration, all in registers:
// the masked p_burn of rows y - 1, y, y + 1 (neighbour columns by shuffles;
// the halo lanes also keep their outer column), lam and glam of the row, the
// eight products glam(v) r(v, d), which go to the accumulators of their
// source cells u = v - Delta_d (rows y - 1, y, y + 1 of this lane's column,
// or of the neighbouring lane's through shuffles).  After row y the
// accumulator of row y - 1 is complete and dL/dp_burn of that row is
// written.  Every load is a coalesced row segment; next row's loads are
// issued before this row is computed.  lam sums d = 0..7 like the other
// kernels; the gather adds the products in a fixed order of its own.
constexpr int kSweepWarps = 4;

// masked p_burn and the mask at (y, x), zero outside the grid
__device__ __forceinline__ float2 sweep_pb(const float* __restrict__ pburn, const float* __restrict__ mask,
                                           int64_t off, int y, int x, int H, int W) {
    if (y < 0 || y >= H || x < 0 || x >= W) return make_float2(0.f, 0.f);
    const int64_t i = off + (int64_t)y * W + x;
    const float m = mask != nullptr ? mask[i] : 0.f;
    const float p = pburn[i];
    return make_float2(mask != nullptr ? p * (1.0f - m) : p, m);
}

// Each lane streams its column through a private ring of kSwDepth rows in
// shared memory, filled by asynchronous copies kSwDepth - 1 rows ahead (no
// lane reads another lane's slots, so only the copy groups need waiting for).
constexpr int kSwDepth = 4;
// one ring slot = one row of the strip, field by field across the lanes (a
// lane's accesses fall on distinct banks)
struct __align__(16) SwSlot {
    float4 ra[32], rb[32];      // rate row of (y, x)
    float pu[32], au[32], ab[32];   // p_un and the incoming adjoints at (y, x)
    float pbn[32], mn[32];      // p_burn and mask at (y + 2, x)
    float pbo[32], mo[32];      // ... and at (y + 2, outer column) for the halo lanes
};

// Issue the copies of target row y into a ring slot: v = the cell index of
// (y, x) (only used when the cell exists), col / col_o whether this lane's
// column and (halo lanes) its outer column lie in the grid, dxo = outer
// column - x.
template <bool MASKED>
__device__ __forceinline__ void sweep_issue(SwSlot& sl, int lane, const float* __restrict__ r,
                                            const float* __restrict__ pun, const float* __restrict__ pburn,
                                            const float* __restrict__ mask, const float* __restrict__ gun_out,
                                            const float* __restrict__ gburn_out, int64_t v, int y, bool col,
                                            bool col_o, int dxo, int H, int W) {
    if (col && (unsigned)y < (unsigned)H) {
        jwf_cp_async16(reinterpret_cast<float*>(&sl.ra[lane]), r + v * 8);
        jwf_cp_async16(reinterpret_cast<float*>(&sl.rb[lane]), r + v * 8 + 4);
        jwf_cp_async4(&sl.pu[lane], pun + v);
        jwf_cp_async4(&sl.au[lane], gun_out + v);
        jwf_cp_async4(&sl.ab[lane], gburn_out + v);
    } else {
        sl.ra[lane] = make_float4(0.f, 0.f, 0.f, 0.f);
        sl.rb[lane] = make_float4(0.f, 0.f, 0.f, 0.f);
        sl.pu[lane] = 0.f;
        sl.au[lane] = 0.f;
        sl.ab[lane] = 0.f;
    }
    const bool row2 = (unsigned)(y + 2) < (unsigned)H;
    const int64_t v2 = v + 2 * (int64_t)W;
    // (the mask fields are written, and read, only by the variant with masks)
    if (col && row2) {
        jwf_cp_async4(&sl.pbn[lane], pburn + v2);
        if constexpr (MASKED) {
            if (mask != nullptr) jwf_cp_async4(&sl.mn[lane], mask + v2);
            else sl.mn[lane] = 0.f;
        }
    } else {
        sl.pbn[lane] = 0.f;
        if constexpr (MASKED) sl.mn[lane] = 0.f;
    }
    if (col_o && row2) {
        jwf_cp_async4(&sl.pbo[lane], pburn + v2 + dxo);
        if constexpr (MASKED) {
            if (mask != nullptr) jwf_cp_async4(&sl.mo[lane], mask + v2 + dxo);
            else sl.mo[lane] = 0.f;
        }
    } else {
        sl.pbo[lane] = 0.f;
        if constexpr (MASKED) sl.mo[lane] = 0.f;
    }
    jwf_cp_async_commit();
}

template <int N>
__device__ __forceinline__ void cp_async_wait_n() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <bool MASKED>
__global__ void __launch_bounds__(kSweepWarps * 32)
k_relaxed_bwd_sweep(const int4* __restrict__ items, int64_t n_items, const int32_t* __restrict__ Hs,
                    const int32_t* __restrict__ Ws, const int64_t* __restrict__ offs,
                    const float* __restrict__ r, const float* __restrict__ pun,
                    const float* __restrict__ pburn, const float* __restrict__ mask,
                    const float* __restrict__ gun_out, const float* __restrict__ gburn_out, float p_continue,
                    float* __restrict__ gun, float* __restrict__ gburn, float* __restrict__ glam,
                    double* __restrict__ partials, uint32_t* __restrict__ counter, double* __restrict__ gpc) {
    __shared__ double red[kSweepWarps];
    __shared__ bool am_last;
    __shared__ SwSlot ring[kSweepWarps][kSwDepth];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double acc = 0.0;
    float accf = 0.f;           // a strip's share of dL/dp_continue, added to acc per strip
    for (int64_t it = (int64_t)blockIdx.x * kSweepWarps + warp; it < n_items; it += (int64_t)gridDim.x * kSweepWarps) {
        const int4 w = items[it];
        const int e = w.x, y0 = w.y, x0 = w.z;
        const int H = Hs[e], W = Ws[e];
        const int64_t off = offs[e];
        const int y1 = min(y0 + JWF_SW_ROWS, H);
        const int x = x0 - 1 + lane;
        const bool out_col = lane >= 1 && lane <= JWF_SW_COLS && x < W;
        // outer column of the halo lanes (their neighbour outside the warp)
        const int xo = lane == 0 ? x - 1 : x + 1;
        const bool edge = lane == 0 || lane == 31;
        // p_burn windows: rows y - 1, y, y + 1 of the target row y
        float2 pa = sweep_pb(pburn, MASKED ? mask : nullptr, off, y0 - 2, x, H, W);
        float2 pb = sweep_pb(pburn, MASKED ? mask : nullptr, off, y0 - 1, x, H, W);
        float2 pc = sweep_pb(pburn, MASKED ? mask : nullptr, off, y0, x, H, W);
        float oa = 0.f, ob = 0.f, oc = 0.f;
        if (edge) {
            oa = sweep_pb(pburn, MASKED ? mask : nullptr, off, y0 - 2, xo, H, W).x;
            ob = sweep_pb(pburn, MASKED ? mask : nullptr, off, y0 - 1, xo, H, W).x;
            oc = sweep_pb(pburn, MASKED ? mask : nullptr, off, y0, xo, H, W).x;
        }
        const int yb = y0 - 1;                            // first target row
        const bool col = x >= 0 && x < W, col_o = edge && xo >= 0 && xo < W;
        // cell indices of (row, x), advanced a row at a time: the row being
        // issued and the target row
        int64_t v_is = off + (int64_t)yb * W + x;
        int64_t v = v_is;
        for (int k = 0; k < kSwDepth - 1; ++k, v_is += W)
            sweep_issue<MASKED>(ring[warp][k], lane, r, pun, pburn, mask, gun_out, gburn_out, v_is, yb + k, col, col_o,
                        xo - x, H, W);
        float g_prev = 0.f, g_cur = 0.f, g_next = 0.f;   // accumulators of rows y - 1, y, y + 1
        float ab_prev = 0.f, m_prev = 0.f;                // a_b and mask of row y - 1
        for (int y = yb; y <= y1; ++y, v += W, v_is += W) {
            const int k = y - yb;
            sweep_issue<MASKED>(ring[warp][(k + kSwDepth - 1) % kSwDepth], lane, r, pun, pburn, mask, gun_out, gburn_out,
                        v_is, y + kSwDepth - 1, col, col_o, xo - x, H, W);
            cp_async_wait_n<kSwDepth - 1>();
            const SwSlot& sl = ring[warp][k % kSwDepth];
            struct {
                float4 ra, rb;
                float pu, au, ab;
            } cur = {sl.ra[lane], sl.rb[lane], sl.pu[lane], sl.au[lane], sl.ab[lane]};
            const bool mk = MASKED && mask != nullptr;
            const float pbn = sl.pbn[lane], mn = mk ? sl.mn[lane] : 0.f;
            const float2 pn = make_float2(mk ? pbn * (1.0f - mn) : pbn, mn);
            const float on = mk ? sl.pbo[lane] * (1.0f - sl.mo[lane]) : sl.pbo[lane];
            // neighbour columns of the window
            float la = __shfl_up_sync(FULL, pa.x, 1), lb = __shfl_up_sync(FULL, pb.x, 1),
                  lc = __shfl_up_sync(FULL, pc.x, 1);
            float ra_ = __shfl_down_sync(FULL, pa.x, 1), rb_ = __shfl_down_sync(FULL, pb.x, 1),
                  rc_ = __shfl_down_sync(FULL, pc.x, 1);
            if (lane == 0) {
                la = oa;
                lb = ob;
                lc = oc;
            }
            if (lane == 31) {
                ra_ = oa;
                rb_ = ob;
                rc_ = oc;
            }
            const float rv[8] = {cur.ra.x, cur.ra.y, cur.ra.z, cur.ra.w, cur.rb.x, cur.rb.y, cur.rb.z, cur.rb.w};
            // sources of directions 0..7: (y, x-1), (y+1, x-1), (y+1, x), (y+1, x+1), (y, x+1), (y-1, x+1),
            // (y-1, x), (y-1, x-1)
            const float src[8] = {lb, lc, pc.x, rc_, rb_, ra_, pa.x, la};
            float lam = 0.f;
#pragma unroll
            for (int d = 0; d < 8; ++d) lam += src[d] * rv[d];
            const bool valid = col && (unsigned)y < (unsigned)H;
            float g = 0.f;
            if (valid) {
                const float em = expf(-lam);
                const float p_ign = -expm1f(-lam);
                const float nb = cur.ab - cur.au;
                const float pe = cur.pu * em;
                g = pe != 0.f ? sat(nb * pe) : 0.f;
                if (out_col && y >= y0 && y < y1) {
                    gun[v] = sat(p_ign != 0.f ? cur.au + nb * p_ign : cur.au);
                    glam[v] = g;
                    if (pb.x != 0.f) accf += cur.ab * pb.x;
                }
            }
            float P[8];
#pragma unroll
            for (int d = 0; d < 8; ++d) P[d] = g * rv[d];
            // products to the source cells: own column (d = 2 -> row y+1, d = 6 -> row y-1); the column
            // to the left gets d = 0, 1, 7 (rows y, y+1, y-1) from its right neighbour, the column to the
            // right gets d = 3, 4, 5 (rows y+1, y, y-1) from its left neighbour
            const float fr0 = __shfl_down_sync(FULL, P[0], 1), fr1 = __shfl_down_sync(FULL, P[1], 1),
                        fr7 = __shfl_down_sync(FULL, P[7], 1);
            const float fl3 = __shfl_up_sync(FULL, P[3], 1), fl4 = __shfl_up_sync(FULL, P[4], 1),
                        fl5 = __shfl_up_sync(FULL, P[5], 1);
            g_prev += P[6];
            g_prev += fr7;
            g_prev += fl5;
            g_cur += fr0;
            g_cur += fl4;
            g_next += P[2];
            g_next += fr1;
            g_next += fl3;
            // row y - 1 is complete
            if (out_col && y - 1 >= y0 && y - 1 < y1) {
                float gb = p_continue != 0.f ? p_continue * ab_prev + g_prev : g_prev;
                if (mk) {
                    const float keep = 1.0f - m_prev;
                    gb = keep != 0.f ? gb * keep : 0.f;
                }
                gburn[v - W] = sat(gb);
            }
            g_prev = g_cur;
            g_cur = g_next;
            g_next = 0.f;
            ab_prev = cur.ab;
            m_prev = pb.y;
            pa = pb;
            pb = pc;
            pc = pn;
            oa = ob;
            ob = oc;
            oc = on;
        }
        jwf_cp_async_wait_all();      // the rows fetched past the strip's end land before the ring is reused
        acc += (double)accf;
        accf = 0.f;
    }
    if (gpc == nullptr) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < kSweepWarps; ++i) s += red[i];
        partials[blockIdx.x] = s;
        __threadfence();
        am_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    double s = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) s += __ldcg(&partials[b]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int i = 0; i < kSweepWarps; ++i) tot += red[i];
        *gpc += tot;
        *counter = 0u;
    }
}
// Two adjoint steps per pass.  The sweep carries the adjoint of step t + 1
// (target row y) and, one row behind, the adjoint of step t (target row
// y - 1): the adjoint of p_burn at row y - 1 after step t + 1's sweep is
// complete once row y has been swept, and it is the incoming adjoint of step
// t at that row, so each rate row is read once for both steps and the
// adjoint between the steps never leaves the chip.  Lane L is column
// x0 - 2 + L: step t + 1 is valid on lanes 1..30 (lanes 0 and 31 also keep
// their outer column's p_burn), step t on lanes 2..29, the strip's output
// columns.  Every cell's arithmetic, and the order of each sum, is that of
// k_relaxed_bwd_sweep, so the adjoints equal two one-step sweeps.
struct __align__(16) Sw2Slot {
    float4 ra[32], rb[32];          // rate row of (y, x)
    float pu1[32], au[32], ab[32];  // p_un before step t + 1 and the incoming adjoints at (y, x)
    float pbn1[32], mn1[32];        // p_burn and mask of step t + 1 at (y + 2, x)
    float pbo1[32], mo1[32];        // ... and at (y + 2, outer column) for the halo lanes
    float pu0[32];                  // p_un before step t at (y - 1, x)
    float pbn0[32], mn0[32];        // p_burn and mask of step t at (y + 1, x)
};
constexpr int kSw2Depth = 3;

template <bool MASKED>
__device__ __forceinline__ void sweep2_issue(Sw2Slot& sl, int lane, const float* __restrict__ r,
                                             const float* __restrict__ pun0, const float* __restrict__ pburn0,
                                             const float* __restrict__ mask0, const float* __restrict__ pun1,
                                             const float* __restrict__ pburn1, const float* __restrict__ mask1,
                                             const float* __restrict__ gun_out, const float* __restrict__ gburn_out,
                                             int64_t v, int y, bool col, bool col_o, int dxo, int H, int W) {
    const bool here = col && (unsigned)y < (unsigned)H;
    if (here) {
        jwf_cp_async16(reinterpret_cast<float*>(&sl.ra[lane]), r + v * 8);
        jwf_cp_async16(reinterpret_cast<float*>(&sl.rb[lane]), r + v * 8 + 4);
        jwf_cp_async4(&sl.pu1[lane], pun1 + v);
        jwf_cp_async4(&sl.au[lane], gun_out + v);
        jwf_cp_async4(&sl.ab[lane], gburn_out + v);
    } else {
        sl.ra[lane] = make_float4(0.f, 0.f, 0.f, 0.f);
        sl.rb[lane] = make_float4(0.f, 0.f, 0.f, 0.f);
        sl.pu1[lane] = 0.f;
        sl.au[lane] = 0.f;
        sl.ab[lane] = 0.f;
    }
    const bool row2 = (unsigned)(y + 2) < (unsigned)H;
    const int64_t v2 = v + 2 * (int64_t)W;
    // (the mask fields are written, and read, only by the variant with masks)
    if (col && row2) {
        jwf_cp_async4(&sl.pbn1[lane], pburn1 + v2);
        if constexpr (MASKED) {
            if (mask1 != nullptr) jwf_cp_async4(&sl.mn1[lane], mask1 + v2);
            else sl.mn1[lane] = 0.f;
        }
    } else {
        sl.pbn1[lane] = 0.f;
        if constexpr (MASKED) sl.mn1[lane] = 0.f;
    }
    if (col_o && row2) {
        jwf_cp_async4(&sl.pbo1[lane], pburn1 + v2 + dxo);
        if constexpr (MASKED) {
            if (mask1 != nullptr) jwf_cp_async4(&sl.mo1[lane], mask1 + v2 + dxo);
            else sl.mo1[lane] = 0.f;
        }
    } else {
        sl.pbo1[lane] = 0.f;
        if constexpr (MASKED) sl.mo1[lane] = 0.f;
    }
    if (col && (unsigned)(y - 1) < (unsigned)H) jwf_cp_async4(&sl.pu0[lane], pun0 + v - W);
    else sl.pu0[lane] = 0.f;
    if (col && (unsigned)(y + 1) < (unsigned)H) {
        jwf_cp_async4(&sl.pbn0[lane], pburn0 + v + W);
        if constexpr (MASKED) {
            if (mask0 != nullptr) jwf_cp_async4(&sl.mn0[lane], mask0 + v + W);
            else sl.mn0[lane] = 0.f;
        }
    } else {
        sl.pbn0[lane] = 0.f;
        if constexpr (MASKED) sl.mn0[lane] = 0.f;
    }
    jwf_cp_async_commit();
}

// Without masks the sweep fits 80 registers: six CTAs an SM instead of five.
template <bool MASKED>
__global__ void __launch_bounds__(kSweepWarps * 32, MASKED ? 5 : 6)
k_relaxed_bwd_sweep2(const int4* __restrict__ items, int64_t n_items, const int32_t* __restrict__ Hs,
                     const int32_t* __restrict__ Ws, const int64_t* __restrict__ offs, const float* __restrict__ r,
                     const float* __restrict__ pun0, const float* __restrict__ pburn0,
                     const float* __restrict__ mask0, const float* __restrict__ pun1,
                     const float* __restrict__ pburn1, const float* __restrict__ mask1,
                     const float* __restrict__ gun_out, const float* __restrict__ gburn_out, float p_continue,
                     float* __restrict__ gun, float* __restrict__ gburn, float* __restrict__ glam0,
                     float* __restrict__ glam1, double* __restrict__ partials, uint32_t* __restrict__ counter,
                     double* __restrict__ gpc) {
    __shared__ double red[kSweepWarps];
    __shared__ bool am_last;
    __shared__ Sw2Slot ring[kSweepWarps][kSw2Depth];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double acc = 0.0;
    float accf = 0.f;
    for (int64_t it = (int64_t)blockIdx.x * kSweepWarps + warp; it < n_items; it += (int64_t)gridDim.x * kSweepWarps) {
        const int4 w = items[it];
        const int e = w.x, y0 = w.y, x0 = w.z;
        const int H = Hs[e], W = Ws[e];
        const int64_t off = offs[e];
        const int y1 = min(y0 + JWF_SW2_ROWS, H);
        const int x = x0 - 2 + lane;
        const bool out_col = lane >= 2 && lane <= JWF_SW2_COLS + 1 && x < W;
        const int xo = lane == 0 ? x - 1 : x + 1;
        const bool edge = lane == 0 || lane == 31;
        const bool col = x >= 0 && x < W, col_o = edge && xo >= 0 && xo < W;
        const int yb = y0 - 2;                            // first target row of step t + 1
        // step t + 1: p_burn window rows y - 1, y, y + 1 (and the halo lanes' outer column)
        float2 pa1 = sweep_pb(pburn1, MASKED ? mask1 : nullptr, off, yb - 1, x, H, W);
        float2 pb1 = sweep_pb(pburn1, MASKED ? mask1 : nullptr, off, yb, x, H, W);
        float2 pc1 = sweep_pb(pburn1, MASKED ? mask1 : nullptr, off, yb + 1, x, H, W);
        float oa = 0.f, ob = 0.f, oc = 0.f;
        if (edge) {
            oa = sweep_pb(pburn1, MASKED ? mask1 : nullptr, off, yb - 1, xo, H, W).x;
            ob = sweep_pb(pburn1, MASKED ? mask1 : nullptr, off, yb, xo, H, W).x;
            oc = sweep_pb(pburn1, MASKED ? mask1 : nullptr, off, yb + 1, xo, H, W).x;
        }
        // step t (target row y - 1): window rows y - 2, y - 1, y
        float2 pa0 = sweep_pb(pburn0, MASKED ? mask0 : nullptr, off, yb - 2, x, H, W);
        float2 pb0 = sweep_pb(pburn0, MASKED ? mask0 : nullptr, off, yb - 1, x, H, W);
        float2 pc0 = sweep_pb(pburn0, MASKED ? mask0 : nullptr, off, yb, x, H, W);
        int64_t v_is = off + (int64_t)yb * W + x;
        int64_t v = v_is;
        for (int k = 0; k < kSw2Depth - 1; ++k, v_is += W)
            sweep2_issue<MASKED>(ring[warp][k], lane, r, pun0, pburn0, mask0, pun1, pburn1, mask1, gun_out, gburn_out, v_is,
                         yb + k, col, col_o, xo - x, H, W);
        float h_prev = 0.f, h_cur = 0.f, h_next = 0.f;   // step t + 1 accumulators, rows y - 1, y, y + 1
        float g_prev = 0.f, g_cur = 0.f, g_next = 0.f;   // step t accumulators, rows y - 2, y - 1, y
        float ab2_prev = 0.f, m1_prev = 0.f;              // incoming a_b and step t + 1 mask of row y - 1
        float au1_prev = 0.f;                             // step t + 1's dL/dp_un of row y - 1
        float ab1_prev = 0.f;                             // step t + 1's dL/dp_burn of row y - 2
        float rp[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};   // rate row of y - 1
        // ring slots: the row being read and the row being fetched (kSw2Depth - 1 ahead)
        int s_use = 0, s_fetch = kSw2Depth - 1;
        for (int y = yb; y <= y1 + 1; ++y, v += W, v_is += W) {
            sweep2_issue<MASKED>(ring[warp][s_fetch], lane, r, pun0, pburn0, mask0, pun1, pburn1, mask1, gun_out,
                                 gburn_out, v_is, y + kSw2Depth - 1, col, col_o, xo - x, H, W);
            cp_async_wait_n<kSw2Depth - 1>();
            const Sw2Slot& sl = ring[warp][s_use];
            s_use = s_use + 1 == kSw2Depth ? 0 : s_use + 1;
            s_fetch = s_fetch + 1 == kSw2Depth ? 0 : s_fetch + 1;
            const float4 ra4 = sl.ra[lane], rb4 = sl.rb[lane];
            const float pu1v = sl.pu1[lane], au2 = sl.au[lane], ab2 = sl.ab[lane];
            const bool mk1 = MASKED && mask1 != nullptr, mk0 = MASKED && mask0 != nullptr;
            const float pbn1 = sl.pbn1[lane], mn1 = mk1 ? sl.mn1[lane] : 0.f;
            const float2 pn1 = make_float2(mk1 ? pbn1 * (1.0f - mn1) : pbn1, mn1);
            const float on = mk1 ? sl.pbo1[lane] * (1.0f - sl.mo1[lane]) : sl.pbo1[lane];
            const float pu0v = sl.pu0[lane];
            const float pbn0 = sl.pbn0[lane], mn0 = mk0 ? sl.mn0[lane] : 0.f;
            const float2 pn0 = make_float2(mk0 ? pbn0 * (1.0f - mn0) : pbn0, mn0);
            const float rv[8] = {ra4.x, ra4.y, ra4.z, ra4.w, rb4.x, rb4.y, rb4.z, rb4.w};
            // ---- step t + 1, target row y ----
            float h1;
            float gun1;
            {
                float la = __shfl_up_sync(FULL, pa1.x, 1), lb = __shfl_up_sync(FULL, pb1.x, 1),
                      lc = __shfl_up_sync(FULL, pc1.x, 1);
                float ra_ = __shfl_down_sync(FULL, pa1.x, 1), rb_ = __shfl_down_sync(FULL, pb1.x, 1),
                      rc_ = __shfl_down_sync(FULL, pc1.x, 1);
                if (lane == 0) {
                    la = oa;
                    lb = ob;
                    lc = oc;
                }
                if (lane == 31) {
                    ra_ = oa;
                    rb_ = ob;
                    rc_ = oc;
                }
                const float src[8] = {lb, lc, pc1.x, rc_, rb_, ra_, pa1.x, la};
                float lam = 0.f;
#pragma unroll
                for (int d = 0; d < 8; ++d) lam += src[d] * rv[d];
                const bool valid = col && (unsigned)y < (unsigned)H;
                h1 = 0.f;
                gun1 = 0.f;
                if (valid) {
                    const float em = expf(-lam);
                    const float p_ign = -expm1f(-lam);
                    const float nb = ab2 - au2;
                    const float pe = pu1v * em;
                    h1 = pe != 0.f ? sat(nb * pe) : 0.f;
                    gun1 = sat(p_ign != 0.f ? au2 + nb * p_ign : au2);
                    if (out_col && y >= y0 && y < y1) {
                        glam1[v] = h1;
                        if (pb1.x != 0.f) accf += ab2 * pb1.x;
                    }
                }
                float P[8];
#pragma unroll
                for (int d = 0; d < 8; ++d) P[d] = h1 * rv[d];
                const float fr0 = __shfl_down_sync(FULL, P[0], 1), fr1 = __shfl_down_sync(FULL, P[1], 1),
                            fr7 = __shfl_down_sync(FULL, P[7], 1);
                const float fl3 = __shfl_up_sync(FULL, P[3], 1), fl4 = __shfl_up_sync(FULL, P[4], 1),
                            fl5 = __shfl_up_sync(FULL, P[5], 1);
                h_prev += P[6];
                h_prev += fr7;
                h_prev += fl5;
                h_cur += fr0;
                h_cur += fl4;
                h_next += P[2];
                h_next += fr1;
                h_next += fl3;
            }
            // step t + 1's dL/dp_burn of row y - 1 is complete
            float ab1 = p_continue != 0.f ? p_continue * ab2_prev + h_prev : h_prev;
            if (mk1) {
                const float keep = 1.0f - m1_prev;
                ab1 = keep != 0.f ? ab1 * keep : 0.f;
            }
            ab1 = sat(ab1);
            // ---- step t, target row y - 1 ----
            {
                const int yy = y - 1;
                float la = __shfl_up_sync(FULL, pa0.x, 1), lb = __shfl_up_sync(FULL, pb0.x, 1),
                      lc = __shfl_up_sync(FULL, pc0.x, 1);
                const float ra_ = __shfl_down_sync(FULL, pa0.x, 1), rb_ = __shfl_down_sync(FULL, pb0.x, 1),
                            rc_ = __shfl_down_sync(FULL, pc0.x, 1);
                const float src[8] = {lb, lc, pc0.x, rc_, rb_, ra_, pa0.x, la};
                float lam = 0.f;
#pragma unroll
                for (int d = 0; d < 8; ++d) lam += src[d] * rp[d];
                const bool valid = col && (unsigned)yy < (unsigned)H;
                float g = 0.f;
                if (valid) {
                    const float em = expf(-lam);
                    const float p_ign = -expm1f(-lam);
                    const float nb = ab1 - au1_prev;
                    const float pe = pu0v * em;
                    g = pe != 0.f ? sat(nb * pe) : 0.f;
                    if (out_col && yy >= y0 && yy < y1) {
                        gun[v - W] = sat(p_ign != 0.f ? au1_prev + nb * p_ign : au1_prev);
                        glam0[v - W] = g;
                        if (pb0.x != 0.f) accf += ab1 * pb0.x;
                    }
                }
                float P[8];
#pragma unroll
                for (int d = 0; d < 8; ++d) P[d] = g * rp[d];
                const float fr0 = __shfl_down_sync(FULL, P[0], 1), fr1 = __shfl_down_sync(FULL, P[1], 1),
                            fr7 = __shfl_down_sync(FULL, P[7], 1);
                const float fl3 = __shfl_up_sync(FULL, P[3], 1), fl4 = __shfl_up_sync(FULL, P[4], 1),
                            fl5 = __shfl_up_sync(FULL, P[5], 1);
                g_prev += P[6];
                g_prev += fr7;
                g_prev += fl5;
                g_cur += fr0;
                g_cur += fl4;
                g_next += P[2];
                g_next += fr1;
                g_next += fl3;
                // step t's dL/dp_burn of row y - 2 is complete
                if (out_col && yy - 1 >= y0 && yy - 1 < y1) {
                    float gb = p_continue != 0.f ? p_continue * ab1_prev + g_prev : g_prev;
                    if (mk0) {
                        const float keep = 1.0f - pa0.y;
                        gb = keep != 0.f ? gb * keep : 0.f;
                    }
                    gburn[v - 2 * (int64_t)W] = sat(gb);
                }
            }
            h_prev = h_cur;
            h_cur = h_next;
            h_next = 0.f;
            g_prev = g_cur;
            g_cur = g_next;
            g_next = 0.f;
            ab2_prev = ab2;
            m1_prev = pb1.y;
            au1_prev = gun1;
            ab1_prev = ab1;
#pragma unroll
            for (int d = 0; d < 8; ++d) rp[d] = rv[d];
            pa1 = pb1;
            pb1 = pc1;
            pc1 = pn1;
            oa = ob;
            ob = oc;
            oc = on;
            pa0 = pb0;
            pb0 = pc0;
            pc0 = pn0;
        }
        jwf_cp_async_wait_all();
        acc += (double)accf;
        accf = 0.f;
    }
    if (gpc == nullptr) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < kSweepWarps; ++i) s += red[i];
        partials[blockIdx.x] = s;
        __threadfence();
        am_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    double s = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) s += __ldcg(&partials[b]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int i = 0; i < kSweepWarps; ++i) tot += red[i];
        *gpc += tot;
        *counter = 0u;
    }
}
}  // namespace

cudaError_t jwf_launch_relaxed_fwd(const jwf_ctx* c, const float* pun, const float* pburn,
                                   const float* mask, float* pun_out, float* pburn_out,
                                   cudaStream_t s) {
    if (c->relaxed_kernel == JWF_RELAXED_PLAIN) {
        k_relaxed_fwd<<<(unsigned)c->n_tiles, JWF_TILE, 0, s>>>(c->d_tiles, c->d_H, c->d_W, c->d_off, c->d_r,
                                                                 pun, pburn, mask, c->P.p_continue, pun_out,
                                                                 pburn_out);
    } else {
        // two persistent CTAs per SM
        static int smem_set[64] = {};
        const size_t smem = fwd_smem_bytes();
        if (c->device < 0 || c->device >= 64) return cudaErrorInvalidDevice;
        if (!smem_set[c->device]) {
            const cudaError_t err =
                cudaFuncSetAttribute(k_relaxed_fwd_tiled, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (err != cudaSuccess) return err;
            smem_set[c->device] = 1;
        }
        int64_t grid = (int64_t)c->num_sms * 2;
        if (grid > c->n_rtiles) grid = c->n_rtiles;
        if (grid < 1) grid = 1;
        k_relaxed_fwd_tiled<<<(unsigned)grid, kFT, smem, s>>>(c->d_rtiles, c->n_rtiles, c->d_H, c->d_W, c->d_off,
                                                               c->d_r, pun, pburn, mask, c->P.p_continue, pun_out,
                                                               pburn_out);
    }
    return cudaGetLastError();
}

cudaError_t jwf_launch_relaxed_fwd2(const jwf_ctx* c, const float* pun, const float* pburn, const float* mask0,
                                    const float* mask1, float* pun1, float* pburn1, float* pun2, float* pburn2,
                                    cudaStream_t s) {
    // persistent CTAs, as many as fit an SM (three with masks, four without)
    const bool masked = mask0 != nullptr || mask1 != nullptr;
    static int per_sm[2][64] = {};
    const size_t smem = masked ? fwd2_smem_bytes<true>() : fwd2_smem_bytes<false>();
    if (c->device < 0 || c->device >= 64) return cudaErrorInvalidDevice;
    int& ps = per_sm[masked ? 1 : 0][c->device];
    if (ps == 0) {
        cudaError_t err =
            masked ? cudaFuncSetAttribute(k_relaxed_fwd2_tiled<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem)
                   : cudaFuncSetAttribute(k_relaxed_fwd2_tiled<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem);
        if (err != cudaSuccess) return err;
        int b = 0;
        err = masked ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_relaxed_fwd2_tiled<true>, kF2T, smem)
                     : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_relaxed_fwd2_tiled<false>, kF2T, smem);
        if (err != cudaSuccess) return err;
        ps = b > 0 ? b : 1;
    }
    int64_t grid = (int64_t)c->num_sms * ps;
    if (grid > c->n_r2tiles) grid = c->n_r2tiles;
    if (grid < 1) grid = 1;
    if (masked)
        k_relaxed_fwd2_tiled<true><<<(unsigned)grid, kF2T, smem, s>>>(
            c->d_r2tiles, c->n_r2tiles, c->d_H, c->d_W, c->d_off, c->d_r, pun, pburn, mask0, mask1,
            c->P.p_continue, pun1, pburn1, pun2, pburn2);
    else
        k_relaxed_fwd2_tiled<false><<<(unsigned)grid, kF2T, smem, s>>>(
            c->d_r2tiles, c->n_r2tiles, c->d_H, c->d_W, c->d_off, c->d_r, pun, pburn, mask0, mask1,
            c->P.p_continue, pun1, pburn1, pun2, pburn2);
    return cudaGetLastError();
}

cudaError_t jwf_launch_relaxed_bwd(jwf_ctx* c, const float* pun, const float* pburn,
                                   const float* mask, const float* gun_out,
                                   const float* gburn_out, float* gun, float* gburn,
                                   float* glam, double* gpc, cudaStream_t s) {
    if (c->relaxed_kernel == JWF_RELAXED_PLAIN) {
        int64_t grid = (int64_t)c->num_sms * 8;
        if (grid > c->n_tiles) grid = c->n_tiles;
        if (grid > c->partial_cap) grid = c->partial_cap;
        k_relaxed_bwd_a<<<(unsigned)grid, JWF_TILE, 0, s>>>(c->d_tiles, c->n_tiles, c->d_H, c->d_W, c->d_off,
                                                             c->d_r, pun, pburn, mask, gun_out, gburn_out,
                                                             gun, glam, c->d_partials, c->d_red_counter, gpc);
        k_relaxed_bwd_b<<<(unsigned)c->n_tiles, JWF_TILE, 0, s>>>(c->d_tiles, c->d_H, c->d_W, c->d_off, c->d_r,
                                                                   mask, gburn_out, glam, c->P.p_continue,
                                                                   gburn);
    } else {
        // column sweeps, grid-stride over the strips with as many CTAs as fit
        // the GPU at once (a fixed grid also keeps the per-CTA partial sums of
        // dL/dp_continue deterministic)
        const bool masked = mask != nullptr;
        static int per_sm[2][64] = {};
        if (c->device < 0 || c->device >= 64) return cudaErrorInvalidDevice;
        int& ps = per_sm[masked ? 1 : 0][c->device];
        if (ps == 0) {
            int b = 0;
            const cudaError_t err =
                masked
                    ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_relaxed_bwd_sweep<true>, kSweepWarps * 32, 0)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_relaxed_bwd_sweep<false>, kSweepWarps * 32,
                                                                    0);
            if (err != cudaSuccess) return err;
            ps = b > 0 ? b : 1;
        }
        int64_t grid = (c->n_stiles + kSweepWarps - 1) / kSweepWarps;
        if (grid > (int64_t)c->num_sms * ps) grid = (int64_t)c->num_sms * ps;
        if (grid > c->partial_cap) grid = c->partial_cap;
        if (grid < 1) grid = 1;
        if (masked)
            k_relaxed_bwd_sweep<true><<<(unsigned)grid, kSweepWarps * 32, 0, s>>>(
                c->d_stiles, c->n_stiles, c->d_H, c->d_W, c->d_off, c->d_r, pun, pburn, mask, gun_out, gburn_out,
                c->P.p_continue, gun, gburn, glam, c->d_partials, c->d_red_counter, gpc);
        else
            k_relaxed_bwd_sweep<false><<<(unsigned)grid, kSweepWarps * 32, 0, s>>>(
                c->d_stiles, c->n_stiles, c->d_H, c->d_W, c->d_off, c->d_r, pun, pburn, mask, gun_out, gburn_out,
                c->P.p_continue, gun, gburn, glam, c->d_partials, c->d_red_counter, gpc);
    }
    return cudaGetLastError();
}

cudaError_t jwf_launch_relaxed_bwd2(jwf_ctx* c, const float* pun0, const float* pburn0, const float* mask0,
                                    const float* pun1, const float* pburn1, const float* mask1,
                                    const float* gun_out, const float* gburn_out, float* gun, float* gburn,
                                    float* glam0, float* glam1, double* gpc, cudaStream_t s) {
    const bool masked = mask0 != nullptr || mask1 != nullptr;
    static int per_sm[2][64] = {};
    if (c->device < 0 || c->device >= 64) return cudaErrorInvalidDevice;
    int& ps = per_sm[masked ? 1 : 0][c->device];
    if (ps == 0) {
        int b = 0;
        const cudaError_t err =
            masked ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_relaxed_bwd_sweep2<true>, kSweepWarps * 32, 0)
                   : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_relaxed_bwd_sweep2<false>, kSweepWarps * 32,
                                                                   0);
        if (err != cudaSuccess) return err;
        ps = b > 0 ? b : 1;
    }
    int64_t grid = (c->n_s2tiles + kSweepWarps - 1) / kSweepWarps;
    if (grid > (int64_t)c->num_sms * ps) grid = (int64_t)c->num_sms * ps;
    if (grid > c->partial_cap) grid = c->partial_cap;
    if (grid < 1) grid = 1;
    if (masked)
        k_relaxed_bwd_sweep2<true><<<(unsigned)grid, kSweepWarps * 32, 0, s>>>(
            c->d_s2tiles, c->n_s2tiles, c->d_H, c->d_W, c->d_off, c->d_r, pun0, pburn0, mask0, pun1, pburn1, mask1,
            gun_out, gburn_out, c->P.p_continue, gun, gburn, glam0, glam1, c->d_partials, c->d_red_counter, gpc);
    else
        k_relaxed_bwd_sweep2<false><<<(unsigned)grid, kSweepWarps * 32, 0, s>>>(
            c->d_s2tiles, c->n_s2tiles, c->d_H, c->d_W, c->d_off, c->d_r, pun0, pburn0, mask0, pun1, pburn1, mask1,
            gun_out, gburn_out, c->P.p_continue, gun, gburn, glam0, glam1, c->d_partials, c->d_red_counter, gpc);
    return cudaGetLastError();
}
