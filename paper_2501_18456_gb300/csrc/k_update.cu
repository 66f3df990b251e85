// Boltzmann-learning step (Eq. 5) fused with the Pearson convergence
// check (Sec. 2.1, "Convergence criterium").
//
// For every site pair i < j and symbols a, b:
//   p_ij = C_ij / M,  p_i = C_ii(a,a) / M                (chain frequencies)
//   J'_ij(a,b) = J_ij(a,b) + lr (f_ij(a,b) - p_ij(a,b))  written to (i,j,a,b)
//                                                        and (j,i,b,a)
//   x = f_ij - f_i f_j,  y = p_ij - p_i p_j              (connected correlations)
// and the sums of x, y, x^2, y^2, xy.  The pair blocks (i, j > i) of site i
// are contiguous in J, f_ij and the counts, so the kernel streams these row
// segments: a CTA takes K whole blocks of one row at a time (K q^2 <= 4096
// elements), each thread loading up to 16 elements of each array with
// independent coalesced loads.  The new blocks are staged in shared memory
// and their transposed (j,i) copies are written in destination order, so
// both writes are coalesced.  On a sparse graph (Sec. 2.2) inactive
// couplings are written as zero.  Each thread adds its x, y terms with
// Kahan-compensated FP32 sums (x and y themselves are FP32, the precision
// of their inputs), the threads are reduced in FP64, and the per-CTA partial
// moments go to a scratch array that a single-CTA kernel sums in a fixed
// order, so the result is deterministic.  The new parameters go to the back
// buffer; the host decides whether to swap it in.
#include "bm_internal.cuh"

#include <math.h>

namespace {

constexpr int kUpdThreads = 256;
constexpr int kUpdElems = 4096;  // elements per tile (K whole q x q blocks)

// K whole blocks per tile: K q^2 <= kUpdElems elements and K q <= kUpdElems / 2
// entries of the f_j, p_j tables (the second bound matters only for q = 1).
__host__ __device__ inline int upd_blocks_per_tile(int q)
{
    return max(1, min(kUpdElems / (q * q), kUpdElems / 2 / q));
}

// Kahan-compensated FP32 accumulator: s - c carries the sum to about one
// ulp whatever the number of terms (each thread adds the terms of its
// elements before the FP64 reduction across threads).
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

template <bool MASKED>  // MASKED: a sparse graph is enabled (inactive couplings written as zero)
__global__ void __launch_bounds__(kUpdThreads) k_update_rows(
    const float *__restrict__ J, float *__restrict__ Jn, const float *__restrict__ fi,
    const float *__restrict__ fij, const int32_t *__restrict__ C, const uint8_t *__restrict__ active, int L, int q,
    float invM, float lr, int want_pearson, long long ntiles, double *__restrict__ partials)
{
    __shared__ float tile[kUpdElems];           // new J of the tile's blocks, (jj, a, b) order
    __shared__ float fj[kUpdElems / 2], pj[kUpdElems / 2];  // f_j(b), p_j(b) of the tile's blocks
    __shared__ float frow[32], prow[32];        // f_i(a), p_i(a)
    const int qq = q * q, K = upd_blocks_per_tile(q);
    const int tid = threadIdx.x;
    // step of kUpdThreads elements in (jj, a, b) and in transposed (jj, b, a) order
    const int djj = kUpdThreads / qq, rem = kUpdThreads - djj * qq, da = rem / q, db = rem - da * q;
    Kahan kx, ky, kxx, kyy, kxy;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        int i, jj0;
        bm_row_tile(t, L, K, i, jj0);
        const int nb = min(K, L - 1 - i - jj0);
        const int nel = nb * qq;
        const int j0 = i + 1 + jj0;
        if (want_pearson) {
            for (int k = tid; k < q; k += kUpdThreads) {
                frow[k] = fi[(size_t)i * q + k];
                prow[k] = (float)C[bm_pair_block(L, i, i) * qq + (size_t)k * (q + 1)] * invM;
            }
            for (int k = tid; k < nb * q; k += kUpdThreads) {
                const int jj = k / q, bb = k - jj * q;
                fj[k] = fi[(size_t)(j0 + jj) * q + bb];
                pj[k] = (float)C[bm_pair_block(L, j0 + jj, j0 + jj) * qq + (size_t)bb * (q + 1)] * invM;
            }
            __syncthreads();
        }
        const size_t baseJ = ((size_t)i * L + j0) * qq, baseC = bm_pair_block(L, i, j0) * qq;
        BmPos3 ps;
        ps.init(tid, q, qq);
#pragma unroll 4
        for (int e = tid; e < nel; e += kUpdThreads) {
            const float f = fij[baseJ + e];
            const float pij = (float)C[baseC + e] * invM;
            // Eq. 5; on a sparse graph an inactive coupling stays zero
            float v = fmaf(lr, f - pij, J[baseJ + e]);
            if (MASKED && !active[baseJ + e]) v = 0.0f;
            Jn[baseJ + e] = v;
            tile[e] = v;
            if (want_pearson) {
                const float x = fmaf(-frow[ps.a], fj[ps.jj * q + ps.b], f);
                const float y = fmaf(-prow[ps.a], pj[ps.jj * q + ps.b], pij);
                kx.add(x);
                ky.add(y);
                kxx.add(x * x);
                kyy.add(y * y);
                kxy.add(x * y);
            }
            ps.step(djj, da, db, q);
        }
        __syncthreads();
        // transposed copies: block (j, i) element u = b q + a is J'_ij(a, b)
        BmPos3 pt;  // (jj, b, a) of destination index d = jj q^2 + b q + a
        pt.init(tid, q, qq);
#pragma unroll 4
        for (int d = tid; d < nel; d += kUpdThreads) {
            Jn[((size_t)(j0 + pt.jj) * L + i) * qq + (d - pt.jj * qq)] = tile[pt.jj * qq + pt.b * q + pt.a];
            pt.step(djj, da, db, q);
        }
        __syncthreads();  // tile and the tables are rewritten by the next tile
    }
    if (!want_pearson) return;
    double m5[5] = {kx.value(), ky.value(), kxx.value(), kyy.value(), kxy.value()};
    __shared__ double red[kUpdThreads / 32][5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m5[k] += __shfl_xor_sync(0xffffffffu, m5[k], o);
    }
    const int lane = tid & 31, warp = tid >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 5; ++k) red[warp][k] = m5[k];
    __syncthreads();
    if (tid < 5) {
        double s = 0.0;
        for (int w = 0; w < kUpdThreads / 32; ++w) s += red[w][tid];
        partials[(size_t)blockIdx.x * 5 + tid] = s;
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

// Sum the per-CTA partials in a fixed order (one CTA, 5 moments): each
// thread adds its strided share of all five with independent loads, then a
// fixed-order tree over the threads.
__global__ void __launch_bounds__(256) k_sum_partials(const double *__restrict__ partials, int nparts, double *out5)
{
    __shared__ double red[5][256];
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int k = threadIdx.x; k < nparts; k += blockDim.x) {
        double v[5];
#pragma unroll
        for (int m = 0; m < 5; ++m) v[m] = partials[(size_t)k * 5 + m];
#pragma unroll
        for (int m = 0; m < 5; ++m) acc[m] += v[m];
    }
#pragma unroll
    for (int m = 0; m < 5; ++m) red[m][threadIdx.x] = acc[m];
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
#pragma unroll
            for (int m = 0; m < 5; ++m) red[m][threadIdx.x] += red[m][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x < 5) out5[threadIdx.x] = red[threadIdx.x][0];
}

}  // namespace

long long bm_update_num_tiles(int L, int q)
{
    return L >= 2 ? bm_row_tiles_upto(L - 1, upd_blocks_per_tile(q)) : 0;
}

int bm_update_num_partials(int L, int q)
{
    long long blocks = bm_update_num_tiles(L, q);
    if (blocks > 608) blocks = 608;  // 4 CTAs per SM on 152 SMs, ~6 tiles each (measured best of 608 and 912)
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
        auto *kern = m->active ? k_update_rows<true> : k_update_rows<false>;
        kern<<<nparts, kUpdThreads, 0, st>>>(m->J, m->J_back, fi, fij, counts, m->active, L, q, invM, lr, want_pearson,
                                             bm_update_num_tiles(L, q), partials);
        BM_CK_LAUNCH("k_update_rows");
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
