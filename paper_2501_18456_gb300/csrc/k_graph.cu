// Sparse interaction graphs (Sec. 2.2, "Training sparse models"): element
// decimation (edDCA) and element activation (eaDCA) of the coupling graph,
// on top of the dense model's parameters.
//
// An element is one coupling entry J_ij(a,b) with i < j (its mirror
// J_ji(b,a) follows it); elements are numbered pair by pair in row order,
// (0,1), (0,2), ..., (1,2), ..., and within a pair a*q + b.  The model keeps
// an activity byte per entry of J's natural layout [i][j][a][b] (kept
// symmetric).  A graph step scores every element, selects exactly n of them
// and applies the change:
//   k_graph_keys    one 64-bit key per element whose ascending order is the
//                   selection order: for decimation the bits of the FP64
//                   score (non-negative, so the bits order like the values;
//                   inactive elements get the largest key), for activation
//                   the complement of those bits (largest score first);
//   k_graph_hist    a 256-bin histogram of one key byte among the keys that
//                   match the bytes already fixed (eight passes, most
//                   significant byte first, give the exact n-th smallest key
//                   T and how many keys equal to T are still to be taken);
//   k_graph_ties    per row tile the number of keys equal to T; an exclusive
//                   scan over the tiles gives each tie its rank in element
//                   order, so ties are taken lowest element first;
//   k_graph_apply   the selected elements: decimation clears their activity
//                   and both coupling entries, activation sets the activity;
//                   the number of changed elements is counted.
// Scores (FP64):
//   decimation  J (p - p'), p' = p e^{-J} / (1 - p + p e^{-J}): the symmetric
//               Kullback-Leibler divergence between the model and the model
//               without the element (p = p_ij(a,b) of the chains);
//   activation  f log(f/p) + (1-f) log((1-f)/(1-p)): the Bernoulli
//               Kullback-Leibler divergence between data and model pair
//               frequencies, the likelihood gain of fitting that coupling.
// Row tiles of K whole q x q blocks (bm_row_tile) keep the reads of J, f_ij
// and the counts contiguous.
#include "bm_internal.cuh"

#include <math.h>

#include <algorithm>
#include <vector>

namespace {

constexpr int kGThreads = 256;
constexpr int kGElems = 4096;  // elements per tile (K whole q x q blocks)

inline int g_blocks_per_tile(int q) { return std::max(1, kGElems / (q * q)); }

__device__ __forceinline__ int g_blocks_per_tile_dev(int q) { return max(1, kGElems / (q * q)); }

// Element number of block (i, j0)'s first entry: pairs before (i, j0) in row order.
__device__ __forceinline__ size_t g_first_element(int L, int i, int j0, int qq)
{
    return ((size_t)i * (2 * L - i - 1) / 2 + (size_t)(j0 - i - 1)) * (size_t)qq;
}

template <int MODE>  // 0: decimation, 1: activation
__global__ void __launch_bounds__(kGThreads) k_graph_keys(const float *__restrict__ J, const float *__restrict__ fij,
                                                          const int32_t *__restrict__ C,
                                                          const uint8_t *__restrict__ active, int L, int q, int M,
                                                          long long ntiles, unsigned long long *__restrict__ keys)
{
    const int qq = q * q, K = g_blocks_per_tile_dev(q);
    const double dM = (double)M;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        int i, jj0;
        bm_row_tile(t, L, K, i, jj0);
        const int j0 = i + 1 + jj0, nel = min(K, L - 1 - i - jj0) * qq;
        const size_t baseJ = ((size_t)i * L + j0) * qq, baseC = bm_pair_block(L, i, j0) * qq;
        const size_t baseE = g_first_element(L, i, j0, qq);
        for (int e = threadIdx.x; e < nel; e += kGThreads) {
            const double p = (double)C[baseC + e] / dM;
            unsigned long long key;
            if (MODE == 0) {
                if (!active[baseJ + e]) {
                    key = ~0ull;
                } else {
                    const double Jx = (double)J[baseJ + e];
                    const double w = p * exp(-Jx);
                    double d = Jx * (p - w / (1.0 - p + w));
                    if (!(d > 0.0)) d = 0.0;
                    key = (unsigned long long)__double_as_longlong(d);
                }
            } else {
                const double f = (double)fij[baseJ + e];
                double A = 0.0;
                if (f > 0.0) A += p > 0.0 ? f * log(f / p) : INFINITY;
                if (f < 1.0) A += p < 1.0 ? (1.0 - f) * log((1.0 - f) / (1.0 - p)) : INFINITY;
                if (!(A > 0.0)) A = 0.0;
                key = ~(unsigned long long)__double_as_longlong(A);
            }
            keys[baseE + e] = key;
        }
    }
}

__global__ void __launch_bounds__(kGThreads) k_graph_hist(const unsigned long long *__restrict__ keys, long long n,
                                                          unsigned long long prefix, unsigned long long pmask,
                                                          int shift, unsigned int *__restrict__ hist)
{
    __shared__ unsigned int hs[256];
    for (int k = threadIdx.x; k < 256; k += blockDim.x) hs[k] = 0;
    __syncthreads();
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const unsigned long long k = keys[e];
        if ((k & pmask) == prefix) atomicAdd(&hs[(k >> shift) & 255u], 1u);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 256; k += blockDim.x)
        if (hs[k]) atomicAdd(&hist[k], hs[k]);
}

__device__ __forceinline__ int block_sum(int v, int *red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    int s = 0;
    for (int w = 0; w < kGThreads / 32; ++w) s += red[w];
    __syncthreads();
    return s;
}

__global__ void __launch_bounds__(kGThreads) k_graph_ties(const unsigned long long *__restrict__ keys, int L, int q,
                                                          long long ntiles, unsigned long long T,
                                                          long long *__restrict__ tile_ties)
{
    __shared__ int red[kGThreads / 32];
    const int qq = q * q, K = g_blocks_per_tile_dev(q);
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        int i, jj0;
        bm_row_tile(t, L, K, i, jj0);
        const int j0 = i + 1 + jj0, nel = min(K, L - 1 - i - jj0) * qq;
        const size_t baseE = g_first_element(L, i, j0, qq);
        int c = 0;
        for (int e = threadIdx.x; e < nel; e += kGThreads) c += keys[baseE + e] == T;
        c = block_sum(c, red);
        if (threadIdx.x == 0) tile_ties[t] = c;
    }
}

template <int MODE>  // 0: decimation, 1: activation
__global__ void __launch_bounds__(kGThreads) k_graph_apply(const unsigned long long *__restrict__ keys, int L, int q,
                                                           long long ntiles, unsigned long long T, long long take_ties,
                                                           const long long *__restrict__ tie_base,
                                                           float *__restrict__ J, uint8_t *__restrict__ active,
                                                           unsigned long long *__restrict__ changed)
{
    __shared__ int wcount[kGThreads / 32];
    const int qq = q * q, K = g_blocks_per_tile_dev(q);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int mine = 0;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        int i, jj0;
        bm_row_tile(t, L, K, i, jj0);
        const int j0 = i + 1 + jj0, nel = min(K, L - 1 - i - jj0) * qq;
        const size_t baseE = g_first_element(L, i, j0, qq);
        long long rank0 = tie_base[t];  // ties of this tile's earlier chunks come after this
        for (int c0 = 0; c0 < nel; c0 += kGThreads) {
            const int e = c0 + threadIdx.x;
            const unsigned long long key = e < nel ? keys[baseE + e] : ~0ull;
            const bool tie = e < nel && key == T;
            // rank of this tie among the tile's ties in element order
            const unsigned int bal = __ballot_sync(0xffffffffu, tie);
            if (lane == 0) wcount[warp] = __popc(bal);
            __syncthreads();
            long long before = rank0;
            int chunk = 0;
            for (int w = 0; w < kGThreads / 32; ++w) {
                if (w < warp) before += wcount[w];
                chunk += wcount[w];
            }
            before += __popc(bal & ((1u << lane) - 1u));
            __syncthreads();
            rank0 += chunk;
            const bool sel = e < nel && (key < T || (tie && before < take_ties));
            if (sel) {
                const int jj = e / qq, w = e - jj * qq, a = w / q, b = w - a * q;
                const size_t x = ((size_t)i * L + j0 + jj) * qq + (size_t)w;
                const size_t y = ((size_t)(j0 + jj) * L + i) * qq + (size_t)b * q + a;
                if (MODE == 0) {
                    mine += active[x] != 0;
                    active[x] = active[y] = 0;
                    J[x] = J[y] = 0.0f;
                } else {
                    mine += active[x] == 0;
                    active[x] = active[y] = 1;
                }
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
    if (lane == 0 && mine) atomicAdd(changed, (unsigned long long)mine);
}

// Activity of every entry: 1 off the diagonal blocks for a fully connected
// graph, 0 everywhere for an empty one (whose couplings are then zero).
__global__ void k_graph_fill(uint8_t *__restrict__ active, float *__restrict__ J, int L, int q, int dense)
{
    const size_t qq = (size_t)q * q, n = (size_t)L * L * qq;
    for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (size_t)gridDim.x * blockDim.x) {
        const size_t blk = x / qq;
        const bool off = blk / L != blk % L;
        active[x] = (dense && off) ? 1 : 0;
        if (!dense) J[x] = 0.0f;
    }
}

long long g_tiles(int L, int q) { return L >= 2 ? bm_row_tiles_upto(L - 1, g_blocks_per_tile(q)) : 0; }

int g_grid(long long ntiles) { return (int)std::max<long long>(1, std::min<long long>(ntiles, 608)); }

// Exact n-th smallest key (n >= 1, at most the number of keys): T and how
// many keys equal to T complete the n smallest.
int g_select(bm_model_s *m, long long nkeys, long long n, unsigned long long *T, long long *take_ties, cudaStream_t st)
{
    unsigned long long prefix = 0, pmask = 0;
    long long need = n;
    unsigned int hist[256];
    const int grid = (int)std::max<long long>(1, std::min<long long>((nkeys + kGThreads - 1) / kGThreads, 1216));
    for (int pass = 0; pass < 8; ++pass) {
        const int shift = 56 - 8 * pass;
        BM_CK(cudaMemsetAsync(m->ghist, 0, 256 * sizeof(unsigned int), st));
        k_graph_hist<<<grid, kGThreads, 0, st>>>(m->gkeys, nkeys, prefix, pmask, shift, m->ghist);
        BM_CK_LAUNCH("k_graph_hist");
        BM_CK(cudaMemcpyAsync(hist, m->ghist, sizeof hist, cudaMemcpyDeviceToHost, st));
        BM_CK(cudaStreamSynchronize(st));
        int d = 0;
        long long acc = 0;
        for (; d < 255 && acc + (long long)hist[d] < need; ++d) acc += hist[d];
        need -= acc;
        prefix |= (unsigned long long)d << shift;
        pmask |= 255ull << shift;
    }
    *T = prefix;
    *take_ties = need;
    return BM_OK;
}

int g_scratch(bm_model_s *m)
{
    const long long ne = (long long)m->L * (m->L - 1) / 2 * m->q * m->q;
    const long long nt = g_tiles(m->L, m->q);
    if (!m->gkeys && ne > 0) BM_CK(cudaMalloc(&m->gkeys, (size_t)ne * sizeof(unsigned long long)));
    if (!m->gtile && nt > 0) BM_CK(cudaMalloc(&m->gtile, (size_t)nt * sizeof(long long)));
    if (!m->ghist) BM_CK(cudaMalloc(&m->ghist, 256 * sizeof(unsigned int) + sizeof(unsigned long long)));
    return BM_OK;
}

// Select the n smallest keys (ties by element number) and apply MODE to them.
template <int MODE>
int g_select_apply(bm_model_s *m, long long n, long long *changed_out, cudaStream_t st)
{
    const int L = m->L, q = m->q;
    const long long ne = (long long)L * (L - 1) / 2 * q * q, nt = g_tiles(L, q);
    unsigned long long T = 0;
    long long take = 0;
    int rc = g_select(m, ne, n, &T, &take, st);
    if (rc != BM_OK) return rc;
    k_graph_ties<<<g_grid(nt), kGThreads, 0, st>>>(m->gkeys, L, q, nt, T, m->gtile);
    BM_CK_LAUNCH("k_graph_ties");
    std::vector<long long> ties((size_t)nt);
    BM_CK(cudaMemcpyAsync(ties.data(), m->gtile, (size_t)nt * sizeof(long long), cudaMemcpyDeviceToHost, st));
    BM_CK(cudaStreamSynchronize(st));
    long long run = 0;
    for (auto &v : ties) {  // exclusive scan in tile (= element) order
        const long long c = v;
        v = run;
        run += c;
    }
    BM_CK(cudaMemcpyAsync(m->gtile, ties.data(), (size_t)nt * sizeof(long long), cudaMemcpyHostToDevice, st));
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(m->ghist + 256);
    BM_CK(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st));
    k_graph_apply<MODE><<<g_grid(nt), kGThreads, 0, st>>>(m->gkeys, L, q, nt, T, take, m->gtile, m->J, m->active, cnt);
    BM_CK_LAUNCH("k_graph_apply");
    unsigned long long changed = 0;
    BM_CK(cudaMemcpyAsync(&changed, cnt, sizeof changed, cudaMemcpyDeviceToHost, st));
    BM_CK(cudaStreamSynchronize(st));  // also: the host copy of the tie ranks is no longer read
    *changed_out = (long long)changed;
    return BM_OK;
}

}  // namespace

extern "C" {

int bm_graph_enable(bm_model m, int dense, void *stream)
{
    if (!m) return bm_fail(BM_EINVAL, "bm_graph_enable: NULL model");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = (size_t)m->L * m->L * m->q * m->q;
    if (!m->active) BM_CK(cudaMalloc(&m->active, n));
    int rc = g_scratch(m);
    if (rc != BM_OK) return rc;
    const int grid = (int)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, 4096));
    k_graph_fill<<<grid, 256, 0, st>>>(m->active, m->J, m->L, m->q, dense ? 1 : 0);
    BM_CK_LAUNCH("k_graph_fill");
    m->n_active = dense ? (long long)m->L * (m->L - 1) / 2 * m->q * m->q : 0;
    if (!dense) {  // the couplings changed: every layout derived from J is stale
        m->mma_current = m->bf_current = m->corr_current = m->jg_current = false;
    }
    return BM_OK;
}

int bm_graph_disable(bm_model m)
{
    if (!m) return bm_fail(BM_EINVAL, "bm_graph_disable: NULL model");
    cudaFree(m->active);
    cudaFree(m->gkeys);
    cudaFree(m->gtile);
    cudaFree(m->ghist);
    m->active = nullptr;
    m->gkeys = nullptr;
    m->gtile = nullptr;
    m->ghist = nullptr;
    m->n_active = 0;
    return BM_OK;
}

int bm_graph_count(bm_model m, long long *n_active, long long *n_elements)
{
    if (!m || !n_active || !n_elements) return bm_fail(BM_EINVAL, "bm_graph_count: NULL argument");
    const long long ne = (long long)m->L * (m->L - 1) / 2 * m->q * m->q;
    *n_elements = ne;
    *n_active = m->active ? m->n_active : ne;
    return BM_OK;
}

int bm_graph_get(bm_model m, uint8_t *active_out, int where, void *stream)
{
    if (!m || !active_out) return bm_fail(BM_EINVAL, "bm_graph_get: NULL argument");
    if (!m->active) return bm_fail(BM_EINVAL, "bm_graph_get: the model has no sparse graph (bm_graph_enable)");
    if (where != BM_HOST && where != BM_DEVICE) return bm_fail(BM_EINVAL, "bm_graph_get: bad where=%d", where);
    const size_t n = (size_t)m->L * m->L * m->q * m->q;
    BM_CK(cudaMemcpyAsync(active_out, m->active, n, where == BM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                          (cudaStream_t)stream));
    if (where == BM_HOST) BM_CK(cudaStreamSynchronize((cudaStream_t)stream));
    return BM_OK;
}

int bm_graph_decimate(bm_model m, const int32_t *counts_dev, int M, long long n, long long *removed_out, void *stream)
{
    if (!m || !counts_dev || !removed_out) return bm_fail(BM_EINVAL, "bm_graph_decimate: NULL argument");
    if (!m->active) return bm_fail(BM_EINVAL, "bm_graph_decimate: the model has no sparse graph (bm_graph_enable)");
    if (M < 1) return bm_fail(BM_EINVAL, "bm_graph_decimate: M=%d < 1", M);
    if (n < 0) return bm_fail(BM_EINVAL, "bm_graph_decimate: n=%lld < 0", n);
    *removed_out = 0;
    n = std::min(n, m->n_active);
    if (n == 0) return BM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const long long nt = g_tiles(m->L, m->q);
    k_graph_keys<0><<<g_grid(nt), kGThreads, 0, st>>>(m->J, nullptr, counts_dev, m->active, m->L, m->q, M, nt, m->gkeys);
    BM_CK_LAUNCH("k_graph_keys");
    long long removed = 0;
    const int rc = g_select_apply<0>(m, n, &removed, st);
    if (rc != BM_OK) return rc;
    m->n_active -= removed;
    m->mma_current = m->bf_current = m->corr_current = m->jg_current = false;  // couplings were zeroed
    *removed_out = removed;
    return BM_OK;
}

int bm_graph_activate(bm_model m, const float *fij_dev, const int32_t *counts_dev, int M, long long n,
                      long long *activated_out, void *stream)
{
    if (!m || !fij_dev || !counts_dev || !activated_out) return bm_fail(BM_EINVAL, "bm_graph_activate: NULL argument");
    if (!m->active) return bm_fail(BM_EINVAL, "bm_graph_activate: the model has no sparse graph (bm_graph_enable)");
    if (M < 1) return bm_fail(BM_EINVAL, "bm_graph_activate: M=%d < 1", M);
    if (n < 0) return bm_fail(BM_EINVAL, "bm_graph_activate: n=%lld < 0", n);
    const long long ne = (long long)m->L * (m->L - 1) / 2 * m->q * m->q;
    *activated_out = 0;
    n = std::min(n, ne);
    if (n == 0) return BM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const long long nt = g_tiles(m->L, m->q);
    k_graph_keys<1><<<g_grid(nt), kGThreads, 0, st>>>(nullptr, fij_dev, counts_dev, nullptr, m->L, m->q, M, nt, m->gkeys);
    BM_CK_LAUNCH("k_graph_keys");
    long long fresh = 0;
    const int rc = g_select_apply<1>(m, n, &fresh, st);
    if (rc != BM_OK) return rc;
    m->n_active += fresh;
    *activated_out = fresh;
    return BM_OK;
}

}  // extern "C"
