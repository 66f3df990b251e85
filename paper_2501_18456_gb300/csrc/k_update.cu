// Boltzmann-learning step (Eq. 5) fused with the Pearson convergence
// check (Sec. 2.1, "Convergence criterium").
//
// One warp per site pair i < j walks the q*q entries of the pair block:
//   p_ij = C_ij / M,  p_i = C_ii(a,a) / M                (chain frequencies)
//   J'_ij(a,b) = J_ij(a,b) + lr (f_ij(a,b) - p_ij(a,b))  written to (i,j,a,b)
//                                                        and (j,i,b,a)
//   x = f_ij - f_i f_j,  y = p_ij - p_i p_j              (connected correlations)
// and accumulates sum x, y, x^2, y^2, xy (x and y themselves are FP32, the
// precision of their inputs): within a pair each lane adds its terms with
// Kahan-compensated FP32 sums, and the pairs are reduced in FP64.  The
// transposed (j,i) copy goes through a per-warp shared-memory tile so both
// writes are coalesced.  Per-CTA partial moments go to a scratch array that
// a single-CTA kernel sums in a fixed order, so the result is
// deterministic.  The new parameters go to the back buffer; the
// host decides whether to swap it in.
#include "bm_internal.cuh"

#include <math.h>

namespace {

constexpr int kUpdWarps = 8;

__device__ __forceinline__ void pair_from_index(long long p, int L, int &i, int &j)
{
    // Rows i hold L-1-i pairs; start(i) = i*(2L-i-1)/2.
    // FP32 estimate of the row; the two loops below make it exact
    const float tL = 2.0f * (float)L - 1.0f;
    int r = (int)floorf((tL - sqrtf(fmaxf(tL * tL - 8.0f * (float)p, 0.0f))) * 0.5f);
    if (r < 0) r = 0;
    if (r > L - 2) r = L - 2;
    auto start = [L](long long rr) { return rr * (2LL * L - rr - 1) / 2; };
    while (r > 0 && start(r) > p) --r;
    while (r < L - 2 && start(r + 1) <= p) ++r;
    i = r;
    j = (int)(p - start(r)) + r + 1;
}

// Kahan-compensated FP32 accumulator: s - c carries the sum to about one
// ulp whatever the number of terms (used for the ~q*q/32 terms a lane adds
// per pair before the FP64 reduction across pairs).
struct Kahan {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x)
    {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

__global__ void __launch_bounds__(kUpdWarps * 32) k_update_pairs(
    const float *__restrict__ J, float *__restrict__ Jn, const float *__restrict__ fi,
    const float *__restrict__ fij, const int32_t *__restrict__ C, int L, int q, float invM,
    float lr, int want_pearson, double *__restrict__ partials)
{
    // per warp: the new (i,j) block for its transposed copy (row stride 33:
    // conflict-free both ways), and the pair's one-site vectors
    __shared__ float tile[kUpdWarps][32 * 33];
    __shared__ float vec[kUpdWarps][4][32];  // p_i(a), p_j(b), f_i(a), f_j(b)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int qq = q * q;
    const long long P = (long long)L * (L - 1) / 2;
    float *tw = tile[warp];
    double sx = 0.0, sy = 0.0, sxx = 0.0, syy = 0.0, sxy = 0.0;
    for (long long p = (long long)blockIdx.x * kUpdWarps + warp; p < P;
         p += (long long)gridDim.x * kUpdWarps) {
        int i, j;
        pair_from_index(p, L, i, j);
        const size_t blk = bm_pair_block(L, i, j) * qq;
        const size_t ij = ((size_t)i * L + j) * qq, ji = ((size_t)j * L + i) * qq;
        if (want_pearson && lane < q) {
            vec[warp][0][lane] = (float)C[bm_pair_block(L, i, i) * qq + (size_t)lane * (q + 1)] * invM;
            vec[warp][1][lane] = (float)C[bm_pair_block(L, j, j) * qq + (size_t)lane * (q + 1)] * invM;
            vec[warp][2][lane] = fi[(size_t)i * q + lane];
            vec[warp][3][lane] = fi[(size_t)j * q + lane];
        }
        __syncwarp();
        Kahan kx, ky, kxx, kyy, kxy;
#pragma unroll 4
        for (int e = lane; e < qq; e += 32) {
            const int a = e / q, b = e - a * q;
            const float f = fij[ij + e];
            const float pij = (float)C[blk + e] * invM;
            const float v = fmaf(lr, f - pij, J[ij + e]);
            Jn[ij + e] = v;
            tw[a * 33 + b] = v;
            if (want_pearson) {
                const float x = fmaf(-vec[warp][2][a], vec[warp][3][b], f);
                const float y = fmaf(-vec[warp][0][a], vec[warp][1][b], pij);
                kx.add(x);
                ky.add(y);
                kxx.add(x * x);
                kyy.add(y * y);
                kxy.add(x * y);
            }
        }
        __syncwarp();
#pragma unroll 4
        for (int e = lane; e < qq; e += 32) {  // (j,i) block: element (b,a) = J'_ij(a,b)
            const int b = e / q, a = e - b * q;
            Jn[ji + e] = tw[a * 33 + b];
        }
        __syncwarp();  // tile and vec are rewritten by the next pair
        if (want_pearson) {
            sx += kx.value();
            sy += ky.value();
            sxx += kxx.value();
            syy += kyy.value();
            sxy += kxy.value();
        }
    }
    if (!want_pearson) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
        sxx += __shfl_xor_sync(0xffffffffu, sxx, o);
        syy += __shfl_xor_sync(0xffffffffu, syy, o);
        sxy += __shfl_xor_sync(0xffffffffu, sxy, o);
    }
    __shared__ double red[kUpdWarps][5];
    if (lane == 0) {
        red[warp][0] = sx;
        red[warp][1] = sy;
        red[warp][2] = sxx;
        red[warp][3] = syy;
        red[warp][4] = sxy;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double s = 0.0;
        for (int w = 0; w < kUpdWarps; ++w) s += red[w][threadIdx.x];
        partials[(size_t)blockIdx.x * 5 + threadIdx.x] = s;
    }
}

__global__ void k_update_fields(const float *__restrict__ h, float *__restrict__ hn,
                                const float *__restrict__ fi, const int32_t *__restrict__ C, int L,
                                int q, float invM, float lr)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= L * q) return;
    const int i = k / q, a = k - i * q;
    const float pa = (float)C[bm_pair_block(L, i, i) * q * q + (size_t)a * q + a] * invM;
    hn[k] = fmaf(lr, fi[k] - pa, h[k]);
}

// Sum the per-CTA partials in a fixed order (one CTA, 5 moments).
__global__ void k_sum_partials(const double *__restrict__ partials, int nparts, double *out5)
{
    __shared__ double red[5][256];
    for (int m = 0; m < 5; ++m) {
        double s = 0.0;
        for (int k = threadIdx.x; k < nparts; k += blockDim.x) s += partials[(size_t)k * 5 + m];
        red[m][threadIdx.x] = s;
    }
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int m = 0; m < 5; ++m) red[m][threadIdx.x] += red[m][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x < 5) out5[threadIdx.x] = red[threadIdx.x][0];
}

}  // namespace

int bm_update_num_partials(int L)
{
    const long long P = (long long)L * (L - 1) / 2;
    long long blocks = (P + kUpdWarps - 1) / kUpdWarps;
    if (blocks > 1216) blocks = 1216;  // 8 CTAs per SM on 152 SMs
    if (blocks < 1) blocks = 1;
    return (int)blocks;
}

int bm_launch_update(bm_model_s *m, const float *fi, const float *fij, const int32_t *counts,
                     int M, float lr, int want_pearson, double *partials, int nparts,
                     double *moments, cudaStream_t st)
{
    const int L = m->L, q = m->q;
    const float invM = 1.0f / (float)M;
    if (L >= 2) {
        k_update_pairs<<<nparts, kUpdWarps * 32, 0, st>>>(m->J, m->J_back, fi, fij, counts, L, q,
                                                          invM, lr, want_pearson, partials);
        BM_CK_LAUNCH("k_update_pairs");
    }
    k_update_fields<<<(L * q + 255) / 256, 256, 0, st>>>(m->h, m->h_back, fi, counts, L, q, invM,
                                                         lr);
    BM_CK_LAUNCH("k_update_fields");
    if (want_pearson) {
        if (L >= 2) {
            k_sum_partials<<<1, 256, 0, st>>>(partials, nparts, moments);
            BM_CK_LAUNCH("k_sum_partials");
        } else {
            BM_CK(cudaMemsetAsync(moments, 0, 5 * sizeof(double), st));
        }
    }
    return BM_OK;
}
