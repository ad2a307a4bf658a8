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

}  // namespace

cudaError_t jwf_launch_relaxed_fwd(const jwf_ctx* c, const float* pun, const float* pburn,
                                   const float* mask, float* pun_out, float* pburn_out,
                                   cudaStream_t s) {
    k_relaxed_fwd<<<(unsigned)c->n_tiles, JWF_TILE, 0, s>>>(c->d_tiles, c->d_H, c->d_W, c->d_off, c->d_r,
                                                             pun, pburn, mask, c->P.p_continue, pun_out,
                                                             pburn_out);
    return cudaGetLastError();
}

cudaError_t jwf_launch_relaxed_bwd(jwf_ctx* c, const float* pun, const float* pburn,
                                   const float* mask, const float* gun_out,
                                   const float* gburn_out, float* gun, float* gburn,
                                   float* glam, double* gpc, cudaStream_t s) {
    int64_t grid = (int64_t)c->num_sms * 8;
    if (grid > c->n_tiles) grid = c->n_tiles;
    if (grid > c->partial_cap) grid = c->partial_cap;
    k_relaxed_bwd_a<<<(unsigned)grid, JWF_TILE, 0, s>>>(c->d_tiles, c->n_tiles, c->d_H, c->d_W, c->d_off,
                                                         c->d_r, pun, pburn, mask, gun_out, gburn_out,
                                                         gun, glam, c->d_partials, c->d_red_counter, gpc);
    k_relaxed_bwd_b<<<(unsigned)c->n_tiles, JWF_TILE, 0, s>>>(c->d_tiles, c->d_H, c->d_W, c->d_off, c->d_r,
                                                               mask, gburn_out, glam, c->P.p_continue, gburn);
    return cudaGetLastError();
}
