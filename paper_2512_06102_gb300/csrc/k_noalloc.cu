// k_noalloc.cu -- jwf_step_relaxed_bwd_noalloc: the relaxed adjoint step for
// a uniform batch, for callers that cannot allocate device memory.
//
// It computes what jwf_step_relaxed_bwd computes (the adjoints of p_un and
// p_burn and dL/dp_continue of one relaxed step) without a context: every
// input and output is a caller pointer, and the scratch the step needs -- the
// plane of dL/dlam between its two passes, the per-block partial sums of the
// p_continue reduction and the counter of the last-block reduction -- lives
// in one file-scope device array, g_noalloc_scratch, sized for at most
// JWF_NOALLOC_MAX_CELLS cells.  Every GPU that loads the library holds that
// array (about 16 MiB) until the process exits.
#include "jwf_internal.cuh"

namespace {

constexpr int kNaThreads = 256;
constexpr int kNaMaxBlocks = 2048;
constexpr size_t kGlamBytes = (size_t)JWF_NOALLOC_MAX_CELLS * sizeof(float);
constexpr size_t kPartialBytes = (size_t)kNaMaxBlocks * sizeof(double);
constexpr size_t kScratchBytes = kGlamBytes + kPartialBytes + 256;

// One array holds the whole scratch: [glam plane | block partials | counter].
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr float kSat = 1e35f;
__device__ __forceinline__ float sat(float x) { return fminf(fmaxf(x, -kSat), kSat); }

__device__ __forceinline__ float pb_of(const float* __restrict__ pburn, const float* __restrict__ mask,
                                       int64_t i) {
    const float p = pburn[i];
    return mask != nullptr ? p * (1.0f - mask[i]) : p;
}

// pass A: dL/dp_un, dL/dlam (to scratch) and the p_continue partial sums
__global__ void __launch_bounds__(kNaThreads)
k_na_bwd_a(int64_t cells, int H, int W, const float* __restrict__ r, const float* __restrict__ pun,
           const float* __restrict__ pburn, const float* __restrict__ mask,
           const float* __restrict__ gun_out, const float* __restrict__ gburn_out,
           float* __restrict__ gun, float* __restrict__ glam, double* __restrict__ partials,
           unsigned int* __restrict__ counter, double* __restrict__ gpc) {
    __shared__ double red[kNaThreads / 32];
    __shared__ bool am_last;
    const int64_t per_env = (int64_t)H * W;
    double acc = 0.0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < cells;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e0 = (v / per_env) * per_env;
        const int local = (int)(v - e0);
        const int y = local / W, x = local - (local / W) * W;
        float lam = 0.f;
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            const int uy = y - jwf_dr(d), ux = x - jwf_dx(d);
            if (uy < 0 || uy >= H || ux < 0 || ux >= W) continue;
            lam += pb_of(pburn, mask, e0 + (int64_t)uy * W + ux) * __ldg(r + v * 8 + d);
        }
        const float em = expf(-lam);
        const float p_ign = -expm1f(-lam);
        const float au = gun_out[v], ab = gburn_out[v];
        const float nb = ab - au;
        const float pe = pun[v] * em;
        gun[v] = sat(p_ign != 0.f ? au + nb * p_ign : au);
        glam[v] = pe != 0.f ? sat(nb * pe) : 0.f;
        const float pbv = pb_of(pburn, mask, v);
        if (pbv != 0.f) acc += (double)(ab * pbv);
    }
    if (gpc == nullptr) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kNaThreads / 32; ++w) s += red[w];
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
        for (int w = 0; w < kNaThreads / 32; ++w) tot += red[w];
        *gpc += tot;
        *counter = 0u;
    }
}

// pass B: dL/dp_burn(u) gathers dL/dlam of the targets u feeds
__global__ void __launch_bounds__(kNaThreads)
k_na_bwd_b(int64_t cells, int H, int W, const float* __restrict__ r, const float* __restrict__ mask,
           const float* __restrict__ gburn_out, const float* __restrict__ glam, float p_continue,
           float* __restrict__ gburn) {
    const int64_t per_env = (int64_t)H * W;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < cells;
         u += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e0 = (u / per_env) * per_env;
        const int local = (int)(u - e0);
        const int y = local / W, x = local - (local / W) * W;
        float g = p_continue != 0.f ? p_continue * gburn_out[u] : 0.f;
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            const int vy = y + jwf_dr(d), vx = x + jwf_dx(d);
            if (vy < 0 || vy >= H || vx < 0 || vx >= W) continue;
            const int64_t v = e0 + (int64_t)vy * W + vx;
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
}

// Device address of the scratch array on the current device.  Looked up on
// every call (a host-side table lookup once the module is loaded), so that a
// context that was destroyed and created again never sees a stale address.
cudaError_t scratch_address(unsigned char** out) {
    void* p = nullptr;
    const cudaError_t err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (err != cudaSuccess) return err;
    *out = static_cast<unsigned char*>(p);
    return cudaSuccess;
}

// [a, a + na) and [b, b + nb) share a byte (null buffers share none)
bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
    if (a == nullptr || b == nullptr) return false;
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + nb && y < x + na;
}

}  // namespace

extern "C" jwf_status jwf_step_relaxed_bwd_noalloc(int32_t n_envs, int32_t H, int32_t W, const float* d_r,
                                                   float p_continue, const float* d_pun,
                                                   const float* d_pburn, const float* d_mask,
                                                   const float* d_gun_out, const float* d_gburn_out,
                                                   float* d_gun, float* d_gburn, double* d_gpc,
                                                   void* stream) {
    if (n_envs < 1 || H < 1 || W < 1) return JWF_EINVAL;
    const int64_t cells = (int64_t)n_envs * H * W;
    if (cells > (int64_t)JWF_NOALLOC_MAX_CELLS) return JWF_EINVAL;
    if (d_r == nullptr || d_pun == nullptr || d_pburn == nullptr || d_gun_out == nullptr ||
        d_gburn_out == nullptr || d_gun == nullptr || d_gburn == nullptr)
        return JWF_EINVAL;
    if (!(p_continue >= 0.f && p_continue <= 1.f)) return JWF_EINVAL;
    // every output must be disjoint from every input and from the other
    // outputs: the two passes read the inputs after the first has written
    const size_t fb = (size_t)cells * sizeof(float);
    const void* ins[] = {d_pun, d_pburn, d_mask, d_gun_out, d_gburn_out, d_r};
    const size_t in_bytes[] = {fb, fb, fb, fb, fb, 8 * fb};
    const void* outs[] = {d_gun, d_gburn, d_gpc};
    const size_t out_bytes[] = {fb, fb, sizeof(double)};
    for (int o = 0; o < 3; ++o) {
        for (int i = 0; i < 6; ++i)
            if (overlaps(outs[o], out_bytes[o], ins[i], in_bytes[i])) return JWF_EINVAL;
        for (int p = o + 1; p < 3; ++p)
            if (overlaps(outs[o], out_bytes[o], outs[p], out_bytes[p])) return JWF_EINVAL;
    }
    unsigned char* base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return JWF_ECUDA;
    float* glam = reinterpret_cast<float*>(base);
    double* partials = reinterpret_cast<double*>(base + kGlamBytes);
    unsigned int* counter = reinterpret_cast<unsigned int*>(base + kGlamBytes + kPartialBytes);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // the reduction counter must start at zero
    if (cudaMemsetAsync(counter, 0, sizeof(unsigned int), s) != cudaSuccess) return JWF_ECUDA;
    int64_t blocks = (cells + kNaThreads - 1) / kNaThreads;
    if (blocks > kNaMaxBlocks) blocks = kNaMaxBlocks;
    k_na_bwd_a<<<(unsigned)blocks, kNaThreads, 0, s>>>(cells, H, W, d_r, d_pun, d_pburn, d_mask, d_gun_out,
                                                         d_gburn_out, d_gun, glam, partials, counter, d_gpc);
    k_na_bwd_b<<<(unsigned)blocks, kNaThreads, 0, s>>>(cells, H, W, d_r, d_mask, d_gburn_out, glam, p_continue,
                                                         d_gburn);
    return cudaGetLastError() == cudaSuccess ? JWF_OK : JWF_ECUDA;
}
