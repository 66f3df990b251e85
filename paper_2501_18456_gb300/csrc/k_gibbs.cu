// Persistent-chain Gibbs sampling on CUDA cores (FP32), and chain
// initialisation.
//
// Method (adabmDCA 2.0, Sec. 2.1 "Monte Carlo estimation of the gradient";
// a sweep proposes every site once, Sec. 3.4): for each chain and each site
// i = 0..L-1 in order, the local field H_i(a) = h_i(a) + sum_{j != i}
// J_ij(a, s_j) (Eq. 1 with all other sites fixed) is formed from the
// current state and s_i is redrawn from p(a) ~ exp(beta H_i(a)).
//
// Mapping: a group of GW lanes (GW = q rounded up to a power of two) owns R
// chains; lane a accumulates H_i(a) for each of its chains.  By the symmetry
// J_ij(a,b) = J_ji(b,a) the gathered vector J_ij(., s_j) is the contiguous
// row J[j][i][s_j][0..q) of the natural layout, so one warp load fetches a
// whole row.  Chain states live in shared memory for the whole launch (all
// nsweeps run in one launch: chains are independent, so no grid-wide
// synchronisation is needed).  J_ii = 0 is enforced at load, so the j = i
// term adds an exact zero and needs no branch.
#include "bm_internal.cuh"

#include <algorithm>

namespace {

__global__ void k_chains_init(uint8_t *__restrict__ s, int M, int L, int q, uint64_t seed)
{
    const size_t n = (size_t)M * L;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (size_t)gridDim.x * blockDim.x) {
        const uint64_t m = t / (size_t)L, i = t % (size_t)L;
        const uint64_t r = bm_u24(seed, m, 0, i, 1);
        s[t] = (uint8_t)((r * (uint64_t)q) >> 24);
    }
}

template <int GW>
__device__ __forceinline__ float group_max(float v)
{
#pragma unroll
    for (int o = GW / 2; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o, GW));
    return v;
}

template <int GW>
__device__ __forceinline__ float group_inclusive_scan(float v, int a)
{
#pragma unroll
    for (int o = 1; o < GW; o <<= 1) {
        const float t = __shfl_up_sync(0xffffffffu, v, o, GW);
        if (a >= o) v += t;
    }
    return v;
}

// GW: lanes per chain group (power of two >= q); R: chains per group.
template <int GW, int R>
__global__ void __launch_bounds__(1024) k_gibbs_simt(const float *__restrict__ h,
                                                     const float *__restrict__ J,
                                                     uint8_t *__restrict__ states, int M, int L,
                                                     int q, int Lp, uint64_t seed,
                                                     uint64_t sweep0, int nsweeps, float beta)
{
    constexpr int G = 32 / GW;  // groups per warp
    extern __shared__ __align__(16) uint8_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane / GW, a = lane % GW;
    const int cpc = (blockDim.x >> 5) * G * R;          // chains per CTA
    const int slot0 = (warp * G + g) * R;                // first chain slot of this group
    const size_t cta0 = (size_t)blockIdx.x * cpc;

    uint8_t *sg = smem + (size_t)slot0 * Lp;             // R rows of Lp bytes
    // Load this group's chains (invalid chains -> zeros, never written back).
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const size_t m = cta0 + slot0 + r;
        for (int k = a; k < Lp; k += GW)
            sg[r * Lp + k] = (m < (size_t)M && k < L) ? states[m * L + k] : 0;
    }
    __syncwarp();

    const int aa = a < q ? a : q - 1;                    // clamp idle lanes to a valid column
    const size_t strideJ = (size_t)L * q * q;            // J[j][i] -> J[j+1][i]
    const unsigned gmask = (GW == 32) ? 0xffffffffu : (((1u << GW) - 1u) << (g * GW));
    const int L4 = L & ~3;

    for (int sw = 0; sw < nsweeps; ++sw) {
        const uint64_t sweep = sweep0 + (uint64_t)sw;
        for (int i = 0; i < L; ++i) {
            float acc[R];
            const float hv = h[(size_t)i * q + aa];
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] = hv;
            // Row base for neighbour j at state b: J + j*strideJ + i*q*q + b*q + a.
            const float *Jc = J + (size_t)i * q * q + aa;
            int j = 0;
            for (; j < L4; j += 4) {
                uint32_t sv[R];
#pragma unroll
                for (int r = 0; r < R; ++r) sv[r] = *reinterpret_cast<const uint32_t *>(sg + r * Lp + j);
                const float *J0 = Jc + (size_t)j * strideJ;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const uint32_t b = (sv[r] >> (8 * k)) & 0xffu;
                        acc[r] += __ldg(J0 + (size_t)k * strideJ + b * q);
                    }
                }
            }
            for (; j < L; ++j) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const uint32_t b = sg[r * Lp + j];
                    acc[r] += __ldg(Jc + (size_t)j * strideJ + b * q);
                }
            }
            // Draw s_i for each chain of the group.
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float e = (a < q) ? beta * acc[r] : -INFINITY;
                const float mx = group_max<GW>(e);
                const float w = (a < q) ? expf(e - mx) : 0.0f;
                const float S = group_inclusive_scan<GW>(w, a);
                const float tot = __shfl_sync(0xffffffffu, S, q - 1, GW);
                const uint64_t m = cta0 + slot0 + r;
                const uint32_t r24 = bm_u24(seed, m, sweep, (uint64_t)i, 0);
                const float t = ((float)r24 * 5.9604644775390625e-8f) * tot;  // u * S_total
                const unsigned bal = __ballot_sync(0xffffffffu, (a < q) && (t < S)) & gmask;
                const int pick = bal ? (__ffs(bal) - 1 - g * GW) : (q - 1);
                if (a == 0) sg[r * Lp + i] = (uint8_t)pick;
            }
            __syncwarp();
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const size_t m = cta0 + slot0 + r;
        if (m < (size_t)M)
            for (int k = a; k < L; k += GW) states[m * L + k] = sg[r * Lp + k];
    }
}

template <int GW, int R>
int launch_gibbs(const bm_model_s *m, bm_chains_s *c, int nsweeps, float beta, int warps,
                 cudaStream_t st)
{
    constexpr int G = 32 / GW;
    const int cpc = warps * G * R;
    const int Lp = (c->L + 15) & ~15;
    const size_t smem = (size_t)cpc * Lp;
    const int grid = (int)((c->M + cpc - 1) / cpc);
    auto kern = k_gibbs_simt<GW, R>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return bm_cuda_fail(e, "cudaFuncSetAttribute(k_gibbs_simt)");
    }
    kern<<<grid, warps * 32, smem, st>>>(m->h, m->J, c->s, c->M, c->L, c->q, Lp, c->seed, c->sweep,
                                          nsweeps, beta);
    BM_CK_LAUNCH("k_gibbs_simt");
    return BM_OK;
}

template <int GW>
int dispatch_r(int R, const bm_model_s *m, bm_chains_s *c, int nsweeps, float beta, int warps,
               cudaStream_t st)
{
    switch (R) {
    case 1: return launch_gibbs<GW, 1>(m, c, nsweeps, beta, warps, st);
    case 2: return launch_gibbs<GW, 2>(m, c, nsweeps, beta, warps, st);
    case 3: return launch_gibbs<GW, 3>(m, c, nsweeps, beta, warps, st);
    default: return launch_gibbs<GW, 4>(m, c, nsweeps, beta, warps, st);
    }
}

}  // namespace

int bm_launch_chains_init(uint8_t *s, int M, int L, int q, uint64_t seed, cudaStream_t st)
{
    const size_t n = (size_t)M * L;
    const int grid = (int)std::min<size_t>((n + 255) / 256, 65535);
    k_chains_init<<<grid, 256, 0, st>>>(s, M, L, q, seed);
    BM_CK_LAUNCH("k_chains_init");
    return BM_OK;
}

// Launch shape: one CTA per SM holding ceil(M / #SM) chains when that fits
// (<= 32 warps, <= 4 chains per lane group), else several waves.
int bm_launch_gibbs_simt(const bm_model_s *m, bm_chains_s *c, int nsweeps, float beta,
                         cudaStream_t st)
{
    const int q = c->q;
    const int GW = q <= 4 ? 4 : q <= 8 ? 8 : q <= 16 ? 16 : 32;
    const int G = 32 / GW;
    const int nsm = m->num_sms > 0 ? m->num_sms : 1;
    const int cps = (c->M + nsm - 1) / nsm;                      // chains per SM
    int R = (cps + 32 * G - 1) / (32 * G);
    R = std::max(1, std::min(4, R));
    int warps = (cps + G * R - 1) / (G * R);
    warps = std::max(1, std::min(32, warps));
    switch (GW) {
    case 4: return dispatch_r<4>(R, m, c, nsweeps, beta, warps, st);
    case 8: return dispatch_r<8>(R, m, c, nsweeps, beta, warps, st);
    case 16: return dispatch_r<16>(R, m, c, nsweeps, beta, warps, st);
    default: return dispatch_r<32>(R, m, c, nsweeps, beta, warps, st);
    }
}
