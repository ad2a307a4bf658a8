// bitplane.cuh -- pieces shared by the resident (k_resident.cu) and tiled
// (k_tiled.cu) discrete steps: the per-warp scratch layout, byte <-> bit-plane
// conversion of four states, and the evaluation of compared (target,
// source) pairs with the rates of Eqs. 1-4.
#pragma once

#include "jwf_internal.cuh"
#include "rate_model.cuh"
#include "step_common.cuh"

namespace {

constexpr int kListCap = 256;      // active cells shared out per warp pass

// Division of a word index by the words per row WW (a grid's or region's row
// length in 32-cell words), by a multiply-high with the rounded-up reciprocal
// m = ceil(2^32 / WW): floor(n m / 2^32) = floor(n / WW) whenever n (m WW -
// 2^32) < 2^32, which holds for the word indices of these kernels (below
// 2^16, with WW <= 64).  A few instructions instead of an integer division.
struct WordDiv {
    uint32_t m;     // 0 for WW == 1
    __device__ __forceinline__ explicit WordDiv(int WW)
        : m(WW == 1 ? 0u : (uint32_t)((0xffffffffull + (unsigned long long)WW) / (unsigned long long)WW)) {}
    __device__ __forceinline__ int div(int n) const { return m == 0u ? n : (int)__umulhi((uint32_t)n, m); }
};
// per warp: item list, ign and out words, pair list (fused variant)
constexpr int kWarpScratch = kListCap + 64 + 256;

// 4 states (one uint32) -> 4-bit mask of the bytes equal to `pattern`
__device__ __forceinline__ uint32_t nib_eq(uint32_t w, uint32_t pattern) {
    const uint32_t m = __vcmpeq4(w, pattern);
    return (((m & 0x01010101u) * 0x01020408u) >> 24) & 0xFu;
}
// 4-bit mask -> 4 bytes of 0 / 1
__device__ __forceinline__ uint32_t nib_spread(uint32_t n) { return (n * 0x00204081u) & 0x01010101u; }

// Fused variant: the candidate cells of list[it0 .. it0+32) are flattened
// into (cell, direction) pairs, one pair per lane per round, so the rate code
// of Eqs. 1-4 runs once per pair rather than once per direction present in
// any lane.  A success sets the cell's bit in ignw.
// (oy, ox): grid coordinates of word 0, bit 0 of the planes (0, 0 for a
// whole env; the region origin for a tile).
template <class Args>
__device__ __forceinline__ void fused_pairs(const Args& a, const RateConsts& K, const uint32_t* list,
                                            uint32_t* plist, uint32_t* ignw, int it0, int n_pass, int base,
                                            int e, int64_t off, int W, int WW, int oy, int ox, uint32_t tt,
                                            uint32_t ep4, int lane) {
    const int it = it0 + lane;
    const uint32_t item = it < n_pass ? list[it] : 0u;
    const uint32_t dm = (item & (1u << 18)) ? (item >> 10) & 0xFFu : 0u;
    const int np = __popc(dm);
    int incl = np;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const int ptotal = __shfl_sync(0xffffffffu, incl, 31);
    int pos = incl - np;
    for (uint32_t rem = dm; rem != 0u; rem &= rem - 1u) plist[pos++] = ((uint32_t)lane << 3) | (__ffs(rem) - 1);
    __syncwarp();
    for (int p = lane; p < ptotal; p += 32) {
        const uint32_t pe = plist[p];
        const int d = (int)(pe & 7u);
        const uint32_t itm = list[it0 + (int)(pe >> 3)];
        const int ol = (int)(itm >> 5) & 31;
        const int j = (int)itm & 31;
        const int ii = base + ol;
        const int ry = WordDiv(WW).div(ii);
        const int yy = oy + ry;
        const int xx = ox + ((ii - ry * WW) << 5) + j;
        if (pair_ignites(a, K, e, off, W, yy, xx, d, tt, ep4)) atomicOr(&ignw[ol], 1u << j);
    }
    __syncwarp();
}

}  // namespace
