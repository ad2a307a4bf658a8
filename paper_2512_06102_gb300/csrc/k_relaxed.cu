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
// 8 B of state out per cell; the adjoint is split in two passes (glam, then
// the transpose gather) so that no cell recomputes a neighbour's lam.
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
// Tiled variant: 2-D tiles of kRH x kRW cells, staged in shared memory by
// asynchronous copies.  Each warp covers 32 consecutive cells of a row, so the
// rate rows (32 B a cell) stream in 1 KB runs.  The adjoint recomputes lam on
// the tile and a one-cell halo, keeps the products glam(v) r(v, d) of that
// region in shared memory ([d][cell], so that the gather reads consecutive
// words), and gathers dL/dp_burn from there: one kernel, no glam round trip,
// each rate row read once (plus the halo's).  Sums run over d = 0..7 in the
// order of the plain kernels (the gather adds rounded products where the
// plain kernel fuses multiply and add).
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

// Adjoint: two persistent CTAs per SM walk the tiles; per tile a CTA stages
// in shared memory (asynchronous copies) the rate rows, p_un and the incoming
// adjoints of the tile and a one-cell halo, and p_burn and the mask of a
// two-cell halo (zero outside the grid, so that a source or target outside
// the grid contributes nothing and the sums need no bounds tests).  One CTA
// computes while the other one's copies are in flight.
constexpr int kBT = 512;                                   // threads of the adjoint CTA
constexpr int kEW = kRW + 2, kEH = kRH + 2, kEN = kEH * kEW;  // tile + 1: glam and rates
constexpr int kPW = kRW + 4, kPH = kRH + 4, kPN = kPH * kPW;  // tile + 2: pb
struct BwdStage {
    float r[kEN * 8];       // rate rows, [cell][d] as in memory
    float pu[kEN], au[kEN], ab[kEN];
    float pb[kPN], m[kPN];  // p_burn and mask; pb becomes (1 - m) p_burn
};
struct BwdSmem {
    BwdStage st;
    float P[8][kEN];        // glam(v) r(v, d), [d][cell] so that the gather reads consecutive words
    double red[kBT / 32];
};
size_t bwd_smem_bytes() { return sizeof(BwdSmem); }

__device__ __forceinline__ void bwd_stage(BwdStage& b, const int4* __restrict__ tiles, int64_t ti,
                                          const int32_t* __restrict__ Hs, const int32_t* __restrict__ Ws,
                                          const int64_t* __restrict__ offs, const float* __restrict__ r,
                                          const float* __restrict__ pun, const float* __restrict__ pburn,
                                          const float* __restrict__ mask, const float* __restrict__ gun_out,
                                          const float* __restrict__ gburn_out) {
    const int4 tl = tiles[ti];
    const int e = tl.x, y0 = tl.y, x0 = tl.z;
    const int H = Hs[e], W = Ws[e];
    const int64_t off = offs[e];
    for (int i = threadIdx.x; i < kEN; i += kBT) {
        const int y = y0 - 1 + i / kEW, x = x0 - 1 + i % kEW;
        if (y < 0 || y >= H || x < 0 || x >= W) continue;
        const int64_t v = off + (int64_t)y * W + x;
        jwf_cp_async16(&b.r[i * 8], r + v * 8);
        jwf_cp_async16(&b.r[i * 8 + 4], r + v * 8 + 4);
        jwf_cp_async4(&b.pu[i], pun + v);
        jwf_cp_async4(&b.au[i], gun_out + v);
        jwf_cp_async4(&b.ab[i], gburn_out + v);
    }
    for (int i = threadIdx.x; i < kPN; i += kBT) {
        const int y = y0 - 2 + i / kPW, x = x0 - 2 + i % kPW;
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

__global__ void __launch_bounds__(kBT)
k_relaxed_bwd_tiled(const int4* __restrict__ tiles, int64_t n_tiles, const int32_t* __restrict__ Hs,
                    const int32_t* __restrict__ Ws, const int64_t* __restrict__ offs,
                    const float* __restrict__ r, const float* __restrict__ pun,
                    const float* __restrict__ pburn, const float* __restrict__ mask,
                    const float* __restrict__ gun_out, const float* __restrict__ gburn_out, float p_continue,
                    float* __restrict__ gun, float* __restrict__ gburn, float* __restrict__ glam,
                    double* __restrict__ partials, uint32_t* __restrict__ counter, double* __restrict__ gpc) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BwdSmem& S = *reinterpret_cast<BwdSmem*>(smem_raw);
    __shared__ bool am_last;
    double acc = 0.0;
    BwdStage& b = S.st;
    for (int64_t ti = blockIdx.x; ti < n_tiles; ti += gridDim.x) {
        bwd_stage(b, tiles, ti, Hs, Ws, offs, r, pun, pburn, mask, gun_out, gburn_out);
        jwf_cp_async_commit();
        const int4 tl = tiles[ti];
        const int e = tl.x, y0 = tl.y, x0 = tl.z;
        const int H = Hs[e], W = Ws[e];
        const int64_t off = offs[e];
        jwf_cp_async_wait_all();
        __syncthreads();
        if (mask != nullptr) {
            for (int i = threadIdx.x; i < kPN; i += kBT) b.pb[i] = b.pb[i] * (1.0f - b.m[i]);
            __syncthreads();
        }
        // glam (and, inside the tile, dL/dp_un) on the tile and its halo
        for (int i = threadIdx.x; i < kEN; i += kBT) {
            const int ly = i / kEW, lx = i - (i / kEW) * kEW;
            const int y = y0 - 1 + ly, x = x0 - 1 + lx;
            float rv[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            float g = 0.f;
            if (y >= 0 && y < H && x >= 0 && x < W) {
                const float4 ra = *reinterpret_cast<const float4*>(&b.r[i * 8]);
                const float4 rb = *reinterpret_cast<const float4*>(&b.r[i * 8 + 4]);
                rv[0] = ra.x; rv[1] = ra.y; rv[2] = ra.z; rv[3] = ra.w;
                rv[4] = rb.x; rv[5] = rb.y; rv[6] = rb.z; rv[7] = rb.w;
                const float pu = b.pu[i], au = b.au[i], ab = b.ab[i];
                float lam = 0.f;
#pragma unroll
                for (int d = 0; d < 8; ++d) lam += b.pb[(ly + 1 - jwf_dr(d)) * kPW + (lx + 1 - jwf_dx(d))] * rv[d];
                const float em = expf(-lam);
                const float p_ign = -expm1f(-lam);
                const float nb = ab - au;
                const float pe = pu * em;
                g = pe != 0.f ? sat(nb * pe) : 0.f;
                if (ly >= 1 && ly <= kRH && lx >= 1 && lx <= kRW) {
                    const int64_t v = off + (int64_t)y * W + x;
                    gun[v] = sat(p_ign != 0.f ? au + nb * p_ign : au);
                    glam[v] = g;
                    const float pbv = b.pb[(ly + 1) * kPW + lx + 1];
                    if (pbv != 0.f) acc += (double)(ab * pbv);
                }
            }
#pragma unroll
            for (int d = 0; d < 8; ++d) S.P[d][i] = g * rv[d];
        }
        __syncthreads();
        // dL/dp_burn(u) = (1 - m(u)) (p_continue a_b(u) + sum_d glam(u + Delta_d) r[u + Delta_d][d])
        for (int j = threadIdx.x; j < kRH * kRW; j += kBT) {
            const int ty = j / kRW, tx = j - (j / kRW) * kRW;
            const int y = y0 + ty, x = x0 + tx;
            if (y >= H || x >= W) continue;
            const int ei = (ty + 1) * kEW + tx + 1;
            const float abu = b.ab[ei];
            float g = p_continue != 0.f ? p_continue * abu : 0.f;
#pragma unroll
            for (int d = 0; d < 8; ++d) g += S.P[d][(ty + 1 + jwf_dr(d)) * kEW + (tx + 1 + jwf_dx(d))];
            if (mask != nullptr) {
                const float keep = 1.0f - b.m[(ty + 2) * kPW + tx + 2];
                g = keep != 0.f ? g * keep : 0.f;
            }
            gburn[off + (int64_t)y * W + x] = sat(g);
        }
        __syncthreads();
    }
    if (gpc == nullptr) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) S.red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kBT / 32; ++w) s += S.red[w];
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
    if ((threadIdx.x & 31) == 0) S.red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < kBT / 32; ++w) tot += S.red[w];
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
        // two persistent CTAs per SM
        static int smem_set[64] = {};
        const size_t smem = bwd_smem_bytes();
        if (c->device < 0 || c->device >= 64) return cudaErrorInvalidDevice;
        if (!smem_set[c->device]) {
            const cudaError_t err =
                cudaFuncSetAttribute(k_relaxed_bwd_tiled, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (err != cudaSuccess) return err;
            smem_set[c->device] = 1;
        }
        int64_t grid = (int64_t)c->num_sms * 2;
        if (grid > c->n_rtiles) grid = c->n_rtiles;
        if (grid > c->partial_cap) grid = c->partial_cap;
        if (grid < 1) grid = 1;
        k_relaxed_bwd_tiled<<<(unsigned)grid, kBT, smem, s>>>(c->d_rtiles, c->n_rtiles, c->d_H, c->d_W, c->d_off,
                                                            c->d_r, pun, pburn, mask, gun_out, gburn_out,
                                                            c->P.p_continue, gun, gburn, glam, c->d_partials,
                                                            c->d_red_counter, gpc);
    }
    return cudaGetLastError();
}
