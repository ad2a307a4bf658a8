// step_common.cuh -- the per-cell and per-pair ignition tests of the discrete
// step (Section 3 "Stochastic update", Eq. 4), shared by the resident, tiled
// and agent step kernels so that all of them draw the same numbers against
// the same probabilities.
#pragma once

#include "jwf_internal.cuh"
#include "rate_model.cuh"

namespace {

// Table variant: does can-burn cell `cell` ignite this step?  dm: bit d set
// when its source in direction d burns.  Draws: slot 0 words -> d 0..3, slot 1
// words -> d 4..7; success iff u < q.  Any success ignites, so the second half
// is skipped once the first has succeeded.
template <class Args>
__device__ __forceinline__ bool ignites(const Args& a, int e, int64_t off, uint32_t cell, uint32_t dm,
                                        uint32_t tt, uint32_t ep4) {
    const float4* q4 = reinterpret_cast<const float4*>(a.q + (off + cell) * 8);
    bool ign = false;
    if (dm & 0x0Fu) {
        const uint4 u = jwf_philox(make_uint4(cell, tt, (uint32_t)e, ep4), a.key0, a.key1);
        const float4 qa = __ldg(q4);
        ign |= ((dm & 1u) && jwf_u24(u.x) < qa.x) || ((dm & 2u) && jwf_u24(u.y) < qa.y) ||
               ((dm & 4u) && jwf_u24(u.z) < qa.z) || ((dm & 8u) && jwf_u24(u.w) < qa.w);
    }
    if (!ign && (dm & 0xF0u)) {
        const uint4 u = jwf_philox(make_uint4(cell, tt, (uint32_t)e, ep4 + 1u), a.key0, a.key1);
        const float4 qb = __ldg(q4 + 1);
        ign |= ((dm & 16u) && jwf_u24(u.x) < qb.x) || ((dm & 32u) && jwf_u24(u.y) < qb.y) ||
               ((dm & 64u) && jwf_u24(u.z) < qb.z) || ((dm & 128u) && jwf_u24(u.w) < qb.w);
    }
    return ign;
}

// Fused variant, one work item: a compared (target, source) pair in
// direction d (pair = true: does the burning source ignite can-burn cell
// (yy, xx) of env e this step?) or a burning cell's remain-burning draw (pair
// = false: does cell (yy, xx) keep burning?).  Both kinds take one Philox
// block (a warp whose items mix the kinds runs it once); a pair's rate of
// Eqs. 1-4 is evaluated on the spot (rate_model.cuh, as the table kernel
// does) and compared with the Philox word of its direction.
template <class Args>
__device__ __forceinline__ bool item_below(const Args& a, const RateConsts& K, int e, int64_t off, int W, int yy,
                                           int xx, bool pair, int d, uint32_t tt, uint32_t ep4) {
    const uint32_t cell = (uint32_t)(yy * W + xx);
    int cv = 0, cu = 0;
    float zv = 0.f, zu = 0.f;
    float2 w2 = make_float2(0.f, 0.f);
    if (pair) {
        const int64_t v = off + cell;
        const int64_t u = off + (int64_t)(yy - jwf_dr(d)) * W + (xx - jwf_dx(d));
        cv = a.cls[v];
        cu = a.cls[u];
        zv = a.dem[v];
        zu = a.dem[u];
        // a wind series is indexed by the step within the episode (held at its last entry)
        const int ts = a.wser_n > 0 ? min((int)tt, a.wser_n - 1) : 0;
        w2 = a.wexp[((int64_t)ts * a.N + e) * 8 + d];
    }
    const uint4 u4 =
        jwf_philox(make_uint4(cell, tt, (uint32_t)e, ep4 + (pair ? (uint32_t)(d >> 2) : 2u)), a.key0, a.key1);
    const uint32_t uw = !pair ? u4.x : (d & 3) == 0 ? u4.x : (d & 3) == 1 ? u4.y : (d & 3) == 2 ? u4.z : u4.w;
    const float u = jwf_u24(uw);
    return pair ? below_prob(u, K.G[cv][cu], zv, zu, {w2.x, w2.y}, d, K) : u < a.p_continue;
}

// Fused variant, one (target, source) pair: does the burning source in
// direction d ignite can-burn cell (yy, xx) of env e this step?
template <class Args>
__device__ __forceinline__ bool pair_ignites(const Args& a, const RateConsts& K, int e, int64_t off, int W, int yy,
                                             int xx, int d, uint32_t tt, uint32_t ep4) {
    return item_below(a, K, e, off, W, yy, xx, true, d, tt, ep4);
}

// Fused variant, up to ILP work items of one thread at once: kind 1 is a
// burning cell's remain-burning draw, kind 2 a compared (target, source)
// pair in direction d, kind 0 no item.  Terrain is loaded for pairs only.  The items' memory loads, Philox blocks and rates are issued
// stage by stage across the items, so that their latencies overlap.  below[k]
// = the item's uniform is below its probability: for a pair the source
// ignites the target (as pair_ignites), for a draw the cell keeps burning.
template <int ILP, class Args>
__device__ __forceinline__ void eval_items(const Args& a, const RateConsts& K, int e, int64_t off, int W,
                                           const int (&yy)[ILP], const int (&xx)[ILP], const int (&kind)[ILP],
                                           const int (&dd)[ILP], uint32_t tt, uint32_t ep4, bool (&below)[ILP]) {
    int cv[ILP], cu[ILP];
    float zv[ILP], zu[ILP];
    float2 w2[ILP];
    uint32_t cell[ILP];
    const int ts = a.wser_n > 0 ? min((int)tt, a.wser_n - 1) : 0;
    const float2* wx = a.wexp + ((int64_t)ts * a.N + e) * 8;
#pragma unroll
    for (int k = 0; k < ILP; ++k) {
        cell[k] = (uint32_t)(yy[k] * W + xx[k]);
        cv[k] = cu[k] = 0;
        zv[k] = zu[k] = 0.f;
        w2[k] = make_float2(0.f, 0.f);
        if (kind[k] == 2) {
            const int d = dd[k];
            const int64_t v = off + cell[k];
            const int64_t u = off + (int64_t)(yy[k] - jwf_dr(d)) * W + (xx[k] - jwf_dx(d));
            cv[k] = a.cls[v];
            cu[k] = a.cls[u];
            zv[k] = a.dem[v];
            zu[k] = a.dem[u];
            w2[k] = wx[d];
        }
    }
    uint32_t uw[ILP];
#pragma unroll
    for (int k = 0; k < ILP; ++k) {
        const bool pair = kind[k] == 2;
        const int d = dd[k];
        const uint4 u4 = jwf_philox(make_uint4(cell[k], tt, (uint32_t)e, ep4 + (pair ? (uint32_t)(d >> 2) : 2u)),
                                    a.key0, a.key1);
        uw[k] = !pair ? u4.x : (d & 3) == 0 ? u4.x : (d & 3) == 1 ? u4.y : (d & 3) == 2 ? u4.z : u4.w;
    }
#pragma unroll
    for (int k = 0; k < ILP; ++k) {
        const float u = jwf_u24(uw[k]);
        below[k] = kind[k] == 2 ? below_prob(u, K.G[cv[k]][cu[k]], zv[k], zu[k], {w2[k].x, w2[k].y}, dd[k], K)
                                : u < a.p_continue;
    }
}

}  // namespace
