// Internal declarations shared by the translation units of libbmdca.so.
// Nothing here is part of the public ABI (include/bmdca.h is).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/bmdca.h"

// ---------------------------------------------------------------------------
// Handles
// ---------------------------------------------------------------------------
struct bm_model_s {
    int L = 0, q = 0;
    int device = 0;
    int engine = BM_ENGINE_AUTO;
    int sampler = BM_SAMPLER_GIBBS;  // update rule of the sweeps (bm_model_set_sampler)
    // Parameters: front buffer is the live model, back buffer receives the
    // next iterate of bm_update (swapped in when the update is applied).
    float *h = nullptr, *J = nullptr;
    float *h_back = nullptr, *J_back = nullptr;
    // Gather layout of the live J: Jg[i][j][b][a] = J_ij(a,b), each (i,j)
    // block padded to bs floats (16-byte aligned blocks).  Read by the
    // CUDA-core forms only; rebuilt lazily (bm_gather_prepare) when stale.
    float *Jg = nullptr;
    int bs = 0;
    bool jg_current = false;
    // Tensor-core layout of the live J: fp16 hi/lo parts, 128 rows per site
    // block (rows (i,a) of the block, zero padded), Kp columns (j,b) (zero
    // padded to a multiple of 64) in 64-column slabs with hi and lo
    // interleaved, and two TMA tensor maps over it (CUtensorMap, 128 bytes
    // each): 256-row boxes of both slabs (two consecutive blocks),
    // 128-row boxes of one slab, and 128-row boxes of both slabs (one
    // block's hi and lo tiles).  Rebuilt lazily when stale.
    void *Jt = nullptr;
    int Kp = 0;
    bool mma_current = false;
    alignas(64) unsigned char tmap_j[128] = {};
    alignas(64) unsigned char tmap_j1[128] = {};
    alignas(64) unsigned char tmap_jp[128] = {};
    // In-block coupling blocks for the two-CTA sweep's corrections: for
    // site block k (B sites, B = the tensor-core block size) and each pair
    // pi > pj of its sites (slot pi*(pi-1)/2 + pj), J_ij(a, b) at
    // Jc[k][slot][b][a] with rows padded to q4 = q rounded up to 4 floats
    // (zeros beyond q and beyond L).  Rebuilt lazily when stale.
    float *Jc = nullptr;
    bool corr_current = false;
    // The same layout with bf16 hi/lo parts (split-precision fields), its
    // 128-row one-slab tensor map, and its staleness flag.
    void *Jt_bf = nullptr;
    bool bf_current = false;
    alignas(64) unsigned char tmap_bf1[128] = {};
    // Small device scratch for flags / reductions (owned).
    int *dflags = nullptr;       // [8] check words; [3] = device error bits (4: wait timeout);
                                 // [4] = a scored sequence held a symbol >= q;
                                 // [5] = |J| beyond fp16 range in the split layout
    double *dred = nullptr;      // reduction partials, capacity red_cap doubles
    size_t red_cap = 0;
    int num_sms = 0;
    // Sparse interaction graph (bm_graph_enable; null: fully connected): the
    // activity of every entry of J's layout [i][j][a][b] (symmetric), the
    // number of active elements i < j, and the selection's scratch (one
    // 64-bit key per element, per-tile tie counts, a 256-bin histogram
    // followed by one 64-bit counter).
    uint8_t *active = nullptr;
    long long n_active = 0;
    unsigned long long *gkeys = nullptr;
    long long *gtile = nullptr;
    unsigned int *ghist = nullptr;
};

struct bm_chains_s {
    int M = 0, L = 0, q = 0;
    int device = 0;
    uint8_t *s = nullptr;  // [M][L]
    uint64_t seed = 0;
    uint64_t sweep = 0;    // Philox sweep word of the next sweep
    uint64_t chain0 = 0;   // global index of chain 0 (shards of a larger ensemble)
    int stats_engine = BM_STATS_AUTO;
    int *derr = nullptr;   // device error word of this handle's kernels
    // Transposed FP8 one-hot of the states for the tensor-core counts
    // (xt_rows x xt_cols bytes, owned) and its TMA tensor map.
    void *xt = nullptr;
    int xt_rows = 0, xt_cols = 0;
    // Partial counts of the tiles split along the chains (owned; int32), their
    // arrival tickets (owned; epoch in the high word) and the last epoch.
    int32_t *ct_ws = nullptr;
    unsigned long long *ct_cnt = nullptr;
    unsigned int ct_epoch = 0;
    alignas(64) unsigned char tmap_a[128] = {};
};

// ---------------------------------------------------------------------------
// Errors (thread-local message, see bm_last_error)
// ---------------------------------------------------------------------------
int bm_fail(int code, const char *fmt, ...);
int bm_cuda_fail(cudaError_t e, const char *what);

#define BM_CK(call)                                              \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return bm_cuda_fail(e_, #call);   \
    } while (0)

#define BM_CK_LAUNCH(name)                                       \
    do {                                                         \
        cudaError_t e_ = cudaGetLastError();                     \
        if (e_ != cudaSuccess) return bm_cuda_fail(e_, name);    \
    } while (0)

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon et al., SC'11): key (seed, 0), counter
// (chain, sweep, site, tag); only output word 0 is needed by the draws.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t bm_philox_word0(uint64_t seed, uint64_t c0, uint64_t c1,
                                                    uint64_t c2, uint64_t c3)
{
    const uint64_t kM0 = 0xD2E7470EE14C6C93ULL, kM1 = 0xCA5A826395121157ULL;
    const uint64_t kW0 = 0x9E3779B97F4A7C15ULL, kW1 = 0xBB67AE8584CAA73BULL;
    uint64_t k0 = seed, k1 = 0;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0hi = __umul64hi(kM0, c0), p0lo = kM0 * c0;
        const uint64_t p1hi = __umul64hi(kM1, c2), p1lo = kM1 * c2;
        const uint64_t x0 = p1hi ^ c1 ^ k0;
        const uint64_t x2 = p0hi ^ c3 ^ k1;
        c0 = x0;
        c1 = p1lo;
        c2 = x2;
        c3 = p0lo;
        k0 += kW0;
        k1 += kW1;
    }
    return c0;
}

// 24-bit uniform numerator of a draw (top 24 bits of word 0).
__device__ __forceinline__ uint32_t bm_u24(uint64_t seed, uint64_t chain, uint64_t sweep,
                                           uint64_t site, uint64_t tag)
{
    return (uint32_t)(bm_philox_word0(seed, chain, sweep, site, tag) >> 40);
}

// Metropolis-Hastings numerators of site `site` (Sec. 2.1): the proposal
// index k = floor(u24(tag 2) * (q-1) / 2^24) in bits 24-31 (the proposed
// symbol is k, or k+1 when k >= the current symbol) and the acceptance
// numerator u24(tag 3) in bits 0-23.
__device__ __forceinline__ uint32_t bm_mh_word(uint64_t seed, uint64_t chain, uint64_t sweep, uint64_t site, int q)
{
    const uint32_t rp = bm_u24(seed, chain, sweep, site, 2), ra = bm_u24(seed, chain, sweep, site, 3);
    const uint32_t k = q > 1 ? (uint32_t)(((uint64_t)rp * (uint64_t)(q - 1)) >> 24) : 0u;
    return (k << 24) | ra;
}

// Metropolis-Hastings decision from the proposed and current symbols'
// fields scaled by beta*log2(e): accept when d >= 0 or u < 2^d, with
// u = (w & 0xffffff) / 2^24 (the hardware base-2 exponential, a few ulp).
__device__ __forceinline__ bool bm_mh_accept(float hp_l2e, float hc_l2e, uint32_t w)
{
    const float d = hp_l2e - hc_l2e;
    float e;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(d));
    return d >= 0.0f || (float)(w & 0xffffffu) * 5.9604644775390625e-8f < e;
}

// Index of the upper-triangle pair block (i <= j).
__host__ __device__ __forceinline__ size_t bm_pair_block(int L, int i, int j)
{
    return (size_t)i * L - (size_t)i * (i - 1) / 2 + (size_t)(j - i);
}

// Row tiles of the upper pair triangle: row i holds the q x q blocks
// (i, j) for j = i+1..L-1, contiguous in J, f_ij and the counts; a tile is
// K whole blocks of one row.  Tiles of rows with n = 1..N blocks:
// sum over n of ceil(n / K).
__host__ __device__ inline long long bm_row_tiles_upto(long long N, int K)
{
    const long long a = N / K, b = N - a * K;
    return (long long)K * a * (a + 1) / 2 + b * (a + 1);
}

// Tile t -> row i and its first block jj0 (rows in order: the rows before
// row i hold T(L-1) - T(L-1-i) tiles); binary search over the rows.
__host__ __device__ inline void bm_row_tile(long long t, int L, int K, int &i, int &jj0)
{
    const long long TL = bm_row_tiles_upto(L - 1, K);
    int lo = 0, hi = L - 2;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (TL - bm_row_tiles_upto(L - 1 - mid, K) <= t) lo = mid;
        else hi = mid - 1;
    }
    i = lo;
    jj0 = (int)(t - (TL - bm_row_tiles_upto(L - 1 - lo, K))) * K;
}

// Position (jj, a, b) of element e = jj q^2 + a q + b, advanced by a fixed
// step (djj, da, db) without divisions (each carry at most one).
struct BmPos3 {
    int jj, a, b;
    __device__ __forceinline__ void init(int e, int q, int qq)
    {
        jj = e / qq;
        const int w = e - jj * qq;
        a = w / q;
        b = w - a * q;
    }
    __device__ __forceinline__ void step(int djj, int da, int db, int q)
    {
        b += db;
        if (b >= q) {
            b -= q;
            ++a;
        }
        a += da;
        if (a >= q) {
            a -= q;
            ++jj;
        }
        jj += djj;
    }
};

// ---------------------------------------------------------------------------
// Kernel launchers (each returns BM_OK or an error code)
// ---------------------------------------------------------------------------
int bm_launch_check_model(const float *h, const float *J, int L, int q, int *dflags,
                          cudaStream_t st);
int bm_launch_check_symbols(const uint8_t *s, size_t n, int q, int *dflag, cudaStream_t st);
int bm_launch_chains_init(uint8_t *s, int M, int L, int q, uint64_t seed, uint64_t chain0, cudaStream_t st);
int bm_gibbs_mma_chains_per_cta(const bm_model_s *m, int M);
int bm_launch_gibbs_mma(bm_model_s *m, bm_chains_s *c, int nsweeps, float beta, cudaStream_t st);
int bm_gibbs_pair_chains_per_cluster(const bm_model_s *m, int M);
int bm_gibbs_pair_waves(const bm_model_s *m, int M);
bool bm_gibbs_pair_tm(const bm_model_s *m);
// Batches of (model, chains) pairs swept by the two-CTA tensor-core kernel
// in one launch over a work list of chain tiles.
struct bm_pair_batch_s;
int bm_pair_batch_create(bm_model_s *const *models, bm_chains_s *const *chains, int count, bm_pair_batch_s **out);
void bm_pair_batch_free(bm_pair_batch_s *b);
int bm_pair_batch_sweep(bm_pair_batch_s *b, int nsweeps, float beta, cudaStream_t st, uint8_t *const *states_override);
int bm_pair_batch_autotune(bm_pair_batch_s *b, cudaStream_t st);
void bm_pair_batch_shape(const bm_pair_batch_s *b, int *nc, int *ctas);
int bm_launch_gibbs_pair(bm_model_s *m, bm_chains_s *c, int nsweeps, float beta, cudaStream_t st);
int bm_gibbs_paired_chains_per_cluster(const bm_model_s *m, int M);
int bm_gibbs_paired_waves(const bm_model_s *m, int M);
int bm_launch_gibbs_paired(bm_model_s *m, bm_chains_s *c, int nsweeps, float beta, cudaStream_t st);
// Tensor-core sweep form for this model and chain count: 2 = two-CTA
// clusters, 1 = one CTA, 0 = CUDA cores (the model's engine, AUTO resolved).
int bm_sweep_form(const bm_model_s *m, int M);
int bm_gather_block_stride(int q);
int bm_launch_build_gather(const float *J, float *Jg, int L, int q, cudaStream_t st);
int bm_launch_gibbs_simt(const bm_model_s *m, bm_chains_s *c, int nsweeps, float beta,
                         cudaStream_t st);
// nsweeps sweeps of the chains with the model's engine (no argument checks).
int bm_sweep_run(bm_model_s *m, bm_chains_s *c, int nsweeps, float beta, cudaStream_t st);
int bm_launch_chain_stats(const uint8_t *s, int M, int L, int q, int32_t *counts,
                          cudaStream_t st);
int bm_launch_chain_stats_mma(const uint8_t *s, int M, int L, int q, int32_t *counts, int elem_bytes,
                              int *err, cudaStream_t st);
int bm_launch_chain_stats_tc(bm_chains_s *c, int32_t *counts, cudaStream_t st);
int bm_launch_seq_weights(const uint8_t *msa, int N, int L, int thr, float *w, int *cnt,
                          double *meff_dev, cudaStream_t st);
// Bit-sliced form (bm_seq_weights): planes is scratch of
// bm_seq_weights_planes_bytes(N, L) bytes.
size_t bm_seq_weights_planes_bytes(int N, int L);
int bm_launch_seq_weights_bs(const uint8_t *msa, int N, int L, int thr, float *w, int *cnt, uint32_t *planes,
                             double *meff_dev, cudaStream_t st);
int bm_launch_data_stats(const uint8_t *msa, const float *w, int N, int L, int q, double alpha,
                         int frac_bits, double meff, float *fi, float *fij,
                         unsigned long long *acc_fi, cudaStream_t st);
int bm_launch_weight_sum(const float *w, int N, double *out2, cudaStream_t st);
int bm_launch_update(bm_model_s *m, const float *fi, const float *fij, const int32_t *counts,
                     int M, float lr, int want_pearson, double *partials, int nparts,
                     double *moments, cudaStream_t st);
int bm_update_num_partials(int L, int q);
// Rebuilds the gather layout Jg from the live J on `st` when it is stale.
int bm_gather_prepare(bm_model_s *m, cudaStream_t st);
int bm_launch_energy(const bm_model_s *m, const uint8_t *seqs, int n, float *E, int *bad, cudaStream_t st);
int bm_launch_energy_gather(const float *h, const float *J, int L, int q, const uint8_t *seqs, int n,
                            float *E, int *bad, cudaStream_t st);
int bm_launch_energy_staged(const bm_model_s *m, const uint8_t *seqs, int n, float *E, int *bad, cudaStream_t st);
int bm_split_prepare(bm_model_s *m, int bf16, cudaStream_t st);
int bm_split_block_sites(int L, int q);
// The in-block coupling layout Jc of the live J (rebuilt when stale).
int bm_corr_prepare(bm_model_s *m, cudaStream_t st);
int bm_launch_fields_simt(const bm_model_s *m, const uint8_t *seqs, int n, float *H, cudaStream_t st);
int bm_launch_fields_tc(bm_model_s *m, const uint8_t *seqs, int n, float *H, int bf16, cudaStream_t st);
int bm_launch_mutant_scan(const float *h, const float *J, int L, int q, const uint8_t *wt,
                          float *dE, cudaStream_t st);
