// Model checks, energy scoring (Sec. 4.3) and single-mutant scans (Sec. 4.4).
#include "bm_internal.cuh"

#include <algorithm>

namespace {

// Flags: bit 0 asymmetric J, bit 1 nonzero J_ii, bit 2 non-finite value.
// The upper pair blocks (i, j > i) are taken in row tiles of K whole blocks
// (contiguous in J); a tile is staged in shared memory and its transposed
// partners (j, i) are read in their own order, so both reads are coalesced.
// Diagonal blocks and h are checked by a grid-stride pass.
constexpr int kChkElems = 4096;

__host__ __device__ inline int chk_blocks_per_tile(int q) { return max(1, kChkElems / (q * q)); }

__global__ void __launch_bounds__(256) k_check_model(const float *__restrict__ h, const float *__restrict__ J, int L,
                                                     int q, long long ntiles, int *flags)
{
    __shared__ float tile[kChkElems];
    const int qq = q * q, K = chk_blocks_per_tile(q);
    const int tid = threadIdx.x;
    int f = 0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + tid; t < (size_t)L * q; t += stride)
        if (!isfinite(h[t])) f |= 4;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + tid; t < (size_t)L * qq; t += stride) {
        const size_t i = t / qq, e = t - i * qq;
        const float v = J[(i * L + i) * qq + e];
        if (!isfinite(v)) f |= 4;
        if (v != 0.0f) f |= 2;
    }
    const int djj = 256 / qq, rem = 256 - djj * qq, da = rem / q, db = rem - da * q;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        int i, jj0;
        bm_row_tile(t, L, K, i, jj0);
        const int nel = min(K, L - 1 - i - jj0) * qq, j0 = i + 1 + jj0;
        const float *src = J + ((size_t)i * L + j0) * qq;
        for (int e = tid; e < nel; e += 256) {
            const float v = src[e];
            tile[e] = v;
            if (!isfinite(v)) f |= 4;
        }
        __syncthreads();
        BmPos3 pt;  // (jj, b, a) of index d = jj q^2 + b q + a in the transposed blocks
        pt.init(tid, q, qq);
        for (int d = tid; d < nel; d += 256) {
            const float w = J[((size_t)(j0 + pt.jj) * L + i) * qq + (d - pt.jj * qq)];
            const float v = tile[pt.jj * qq + pt.b * q + pt.a];
            if (!isfinite(w)) f |= 4;
            else if (isfinite(v) && !(v == w)) f |= 1;
            pt.step(djj, da, db, q);
        }
        __syncthreads();  // the tile is rewritten by the next one
    }
    f = __reduce_or_sync(0xffffffffu, f);
    if (f && (tid & 31) == 0) atomicOr(flags, f);
}

__global__ void k_check_symbols(const uint8_t *__restrict__ s, size_t n, int q, int *flag)
{
    int bad = 0;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (size_t)gridDim.x * blockDim.x)
        bad |= (s[t] >= q);
    if (bad) atomicOr(flag, 1);
}

// Energy E(s) = -sum_i h_i(s_i) - sum_{i<j} J_ij(s_i, s_j): one warp per
// sequence, lanes stride over j for each i; FP32 accumulation, warp sum.
__global__ void __launch_bounds__(256) k_energy(const float *__restrict__ h,
                                                const float *__restrict__ J, int L, int q,
                                                const uint8_t *__restrict__ S, int n,
                                                float *__restrict__ E, int *bad)
{
    extern __shared__ uint8_t sst[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nw = blockDim.x >> 5;
    uint8_t *s = sst + (size_t)warp * L;
    const size_t qq = (size_t)q * q;
    for (long long k = (long long)blockIdx.x * nw + warp; k < n; k += (long long)gridDim.x * nw) {
        bool inval = false;
        for (int t = lane; t < L; t += 32) {
            const uint8_t v = S[(size_t)k * L + t];
            inval |= v >= q;
            s[t] = v;
        }
        if (__any_sync(0xffffffffu, inval) && lane == 0) atomicOr(bad, 1);
        __syncwarp();
        float acc = 0.0f;
        for (int i = 0; i < L; ++i) {
            const int si = s[i];
            if (si >= q) continue;  // a symbol >= q contributes nothing (flagged above)
            if (lane == 0) acc -= h[(size_t)i * q + si];
            const float *row = J + ((size_t)i * L) * qq + (size_t)si * q;
            for (int j = i + 1 + lane; j < L; j += 32)
                if (s[j] < q) acc -= __ldg(row + (size_t)j * qq + s[j]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) E[k] = acc;
        __syncwarp();
    }
}

// dE(i,a) = -(H_i(a) - H_i(wt_i)), H_i(a) = h_i(a) + sum_{j != i} J_ij(a, wt_j):
// one warp per site, lane = a; J_ij(a, b) read as the contiguous row
// J[j][i][b][.] (symmetry), the j = i term is an exact zero.
__global__ void k_mutant_scan(const float *__restrict__ h, const float *__restrict__ J, int L,
                              int q, const uint8_t *__restrict__ wt, float *__restrict__ dE)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= L) return;
    const int i = warp;
    const int aa = lane < q ? lane : q - 1;
    const size_t qq = (size_t)q * q;
    float H = h[(size_t)i * q + aa];
    for (int j = 0; j < L; ++j) H += __ldg(J + ((size_t)j * L + i) * qq + (size_t)wt[j] * q + aa);
    const float Hw = __shfl_sync(0xffffffffu, H, wt[i]);
    if (lane < q) dE[(size_t)i * q + lane] = (lane == wt[i]) ? 0.0f : -(H - Hw);
}

}  // namespace

int bm_launch_check_model(const float *h, const float *J, int L, int q, int *dflags,
                          cudaStream_t st)
{
    BM_CK(cudaMemsetAsync(dflags, 0, sizeof(int), st));
    const long long ntiles = L >= 2 ? bm_row_tiles_upto(L - 1, chk_blocks_per_tile(q)) : 0;
    const int grid = (int)std::max<long long>(1, std::min<long long>(std::max<long long>(ntiles, (long long)L * q * q / 256 + 1), 1216));
    k_check_model<<<grid, 256, 0, st>>>(h, J, L, q, ntiles, dflags);
    BM_CK_LAUNCH("k_check_model");
    return BM_OK;
}

int bm_launch_check_symbols(const uint8_t *s, size_t n, int q, int *dflag, cudaStream_t st)
{
    BM_CK(cudaMemsetAsync(dflag, 0, sizeof(int), st));
    if (n == 0) return BM_OK;
    const int grid = (int)std::min<size_t>((n + 255) / 256, 4096);
    k_check_symbols<<<grid, 256, 0, st>>>(s, n, q, dflag);
    BM_CK_LAUNCH("k_check_symbols");
    return BM_OK;
}

int bm_launch_energy_gather(const float *h, const float *J, int L, int q, const uint8_t *seqs, int n,
                            float *E, int *bad, cudaStream_t st)
{
    if (n == 0) return BM_OK;
    const int warps = 8;
    const int grid = (int)std::min<long long>(((long long)n + warps - 1) / warps, 152LL * 16);
    k_energy<<<grid, warps * 32, (size_t)warps * L, st>>>(h, J, L, q, seqs, n, E, bad);
    BM_CK_LAUNCH("k_energy");
    return BM_OK;
}

int bm_launch_mutant_scan(const float *h, const float *J, int L, int q, const uint8_t *wt,
                          float *dE, cudaStream_t st)
{
    const int threads = 256;
    const int grid = (L * 32 + threads - 1) / threads;
    k_mutant_scan<<<grid, threads, 0, st>>>(h, J, L, q, wt, dE);
    BM_CK_LAUNCH("k_mutant_scan");
    return BM_OK;
}

// Large batches use the staged form (one pass over J per CTA amortised over
// up to 1024 sequences), smaller ones gather J rows through the caches.  The
// staged form costs about one pass over J whatever the batch, the gather form
// grows with n*L^2: measured crossovers lie near n*L = 3.3e6 (about 8k
// sequences at L = 400, 13k at L = 256, 20k at L = 120).
int bm_launch_energy(const bm_model_s *m, const uint8_t *seqs, int n, float *E, int *bad, cudaStream_t st)
{
    const bool staged = (double)n * m->L >= 3.3e6;
    if (staged && bm_launch_energy_staged(m, seqs, n, E, bad, st) == BM_OK) return BM_OK;
    return bm_launch_energy_gather(m->h, m->J, m->L, m->q, seqs, n, E, bad, st);
}
