// C ABI of libbmdca.so (declared in include/bmdca.h): argument checks,
// handle management and dispatch to the kernels.
#include "bm_internal.cuh"

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>

namespace {
thread_local char g_err[512] = "";

cudaMemcpyKind copy_kind(int src_where, int dst_where)
{
    if (src_where == BM_HOST) return dst_where == BM_HOST ? cudaMemcpyHostToHost : cudaMemcpyHostToDevice;
    return dst_where == BM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
}

bool valid_where(int w) { return w == BM_HOST || w == BM_DEVICE; }

constexpr int kMaxSweepsPerLaunch = 64;

void free_model(bm_model_s *m)
{
    if (!m) return;
    cudaFree(m->h);
    cudaFree(m->J);
    cudaFree(m->h_back);
    cudaFree(m->J_back);
    cudaFree(m->Jg);
    cudaFree(m->Jt);
    cudaFree(m->Jt_bf);
    cudaFree(m->Jc);
    cudaFree(m->dflags);
    cudaFree(m->dred);
    cudaFree(m->active);
    cudaFree(m->gkeys);
    cudaFree(m->gtile);
    cudaFree(m->ghist);
    delete m;
}
}  // namespace

int bm_fail(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

int bm_cuda_fail(cudaError_t e, const char *what)
{
    cudaGetLastError();  // clear a non-sticky error so the next call starts clean
    return bm_fail(e == cudaErrorMemoryAllocation ? BM_ENOMEM : BM_ECUDA, "%s: %s", what,
                   cudaGetErrorString(e));
}

extern "C" {

const char *bm_version(void) { return "bmdca-gb300 0.1"; }

const char *bm_last_error(void) { return g_err; }

int bm_potts_load(const float *h, const float *J, int L, int q, int where, void *stream,
                  bm_model *out)
{
    if (!out) return bm_fail(BM_EINVAL, "bm_potts_load: out is NULL");
    *out = nullptr;
    if (!h || !J) return bm_fail(BM_EINVAL, "bm_potts_load: h or J is NULL");
    if (L < 1 || L > 4096) return bm_fail(BM_EINVAL, "bm_potts_load: L=%d out of [1,4096]", L);
    if (q < 1 || q > 32) return bm_fail(BM_EINVAL, "bm_potts_load: q=%d out of [1,32]", q);
    if (!valid_where(where)) return bm_fail(BM_EINVAL, "bm_potts_load: bad where=%d", where);
    cudaStream_t st = (cudaStream_t)stream;
    bm_model_s *m = new (std::nothrow) bm_model_s();
    if (!m) return bm_fail(BM_ENOMEM, "bm_potts_load: host allocation failed");
    m->L = L;
    m->q = q;
    const size_t nh = (size_t)L * q, nJ = (size_t)L * L * q * q;
    cudaError_t e;
#define LOAD_CK(call)                                  \
    do {                                               \
        e = (call);                                    \
        if (e != cudaSuccess) {                        \
            int rc_ = bm_cuda_fail(e, #call);          \
            free_model(m);                             \
            return rc_;                                \
        }                                              \
    } while (0)
    LOAD_CK(cudaGetDevice(&m->device));
    LOAD_CK(cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, m->device));
    LOAD_CK(cudaMalloc(&m->h, nh * sizeof(float)));
    LOAD_CK(cudaMalloc(&m->J, nJ * sizeof(float)));
    LOAD_CK(cudaMalloc(&m->h_back, nh * sizeof(float)));
    LOAD_CK(cudaMalloc(&m->J_back, nJ * sizeof(float)));
    m->bs = bm_gather_block_stride(q);
    LOAD_CK(cudaMalloc(&m->Jg, (size_t)L * L * m->bs * sizeof(float)));
    LOAD_CK(cudaMalloc(&m->dflags, 8 * sizeof(int)));
    LOAD_CK(cudaMemsetAsync(m->dflags, 0, 8 * sizeof(int), st));
    m->red_cap = (size_t)bm_update_num_partials(L, q) * 5 + 8;
    LOAD_CK(cudaMalloc(&m->dred, m->red_cap * sizeof(double)));
    LOAD_CK(cudaMemcpyAsync(m->h, h, nh * sizeof(float), copy_kind(where, BM_DEVICE), st));
    LOAD_CK(cudaMemcpyAsync(m->J, J, nJ * sizeof(float), copy_kind(where, BM_DEVICE), st));
    LOAD_CK(cudaMemsetAsync(m->J_back, 0, nJ * sizeof(float), st));
    LOAD_CK(cudaMemsetAsync(m->h_back, 0, nh * sizeof(float), st));
    int rc = bm_launch_check_model(m->h, m->J, L, q, m->dflags, st);
    if (rc != BM_OK) {
        free_model(m);
        return rc;
    }
    int flags = 0;
    LOAD_CK(cudaMemcpyAsync(&flags, m->dflags, sizeof(int), cudaMemcpyDeviceToHost, st));
    LOAD_CK(cudaStreamSynchronize(st));
#undef LOAD_CK
    if (flags & 4) {
        free_model(m);
        return bm_fail(BM_ENUMERIC, "bm_potts_load: NaN or Inf in h or J");
    }
    if (flags & 1) {
        free_model(m);
        return bm_fail(BM_EINVAL, "bm_potts_load: J is not symmetric (J[i][j][a][b] != J[j][i][b][a])");
    }
    if (flags & 2) {
        free_model(m);
        return bm_fail(BM_EINVAL, "bm_potts_load: J[i][i] must be zero");
    }
    rc = bm_launch_build_gather(m->J, m->Jg, L, q, st);
    if (rc != BM_OK) {
        free_model(m);
        return rc;
    }
    m->jg_current = true;
    *out = m;
    return BM_OK;
}

int bm_potts_free(bm_model m)
{
    free_model(m);
    return BM_OK;
}

int bm_potts_get(bm_model m, float *h, float *J, int where, void *stream)
{
    if (!m) return bm_fail(BM_EINVAL, "bm_potts_get: NULL model");
    if (!valid_where(where)) return bm_fail(BM_EINVAL, "bm_potts_get: bad where=%d", where);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nh = (size_t)m->L * m->q, nJ = (size_t)m->L * m->L * m->q * m->q;
    if (h) BM_CK(cudaMemcpyAsync(h, m->h, nh * sizeof(float), copy_kind(BM_DEVICE, where), st));
    if (J) BM_CK(cudaMemcpyAsync(J, m->J, nJ * sizeof(float), copy_kind(BM_DEVICE, where), st));
    return BM_OK;
}

int bm_potts_set(bm_model m, const float *h, const float *J, int where, void *stream)
{
    if (!m) return bm_fail(BM_EINVAL, "bm_potts_set: NULL model");
    if (!valid_where(where)) return bm_fail(BM_EINVAL, "bm_potts_set: bad where=%d", where);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nh = (size_t)m->L * m->q, nJ = (size_t)m->L * m->L * m->q * m->q;
    if (h) BM_CK(cudaMemcpyAsync(m->h, h, nh * sizeof(float), copy_kind(where, BM_DEVICE), st));
    if (J) {
        BM_CK(cudaMemcpyAsync(m->J, J, nJ * sizeof(float), copy_kind(where, BM_DEVICE), st));
        m->mma_current = false;
        m->bf_current = false;
        m->corr_current = false;
        m->jg_current = false;
    }
    return BM_OK;
}

int bm_device_status(bm_model m, void *stream)
{
    if (!m) return bm_fail(BM_EINVAL, "bm_device_status: NULL model");
    cudaStream_t st = (cudaStream_t)stream;
    int word[3] = {0, 0, 0};
    BM_CK(cudaMemcpyAsync(word, m->dflags + 3, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
    BM_CK(cudaStreamSynchronize(st));
    if (word[0] || word[1] || word[2]) BM_CK(cudaMemsetAsync(m->dflags + 3, 0, 3 * sizeof(int), st));
    if (word[0]) return bm_fail(BM_ETIMEOUT, "device wait timed out in a Gibbs launch (error word 0x%x)", word[0]);
    if (word[1]) return bm_fail(BM_EINVAL, "a scored sequence held a symbol >= q (it contributed nothing)");
    if (word[2])
        return bm_fail(BM_ENUMERIC, "a coupling exceeds the fp16 range (|J| > 65504) of the tensor-core "
                                    "sweep and fp16 fields; their results are invalid (use BM_ENGINE_SIMT)");
    return BM_OK;
}

int bm_potts_shape(bm_model m, int *L, int *q)
{
    if (!m) return bm_fail(BM_EINVAL, "bm_potts_shape: NULL model");
    if (L) *L = m->L;
    if (q) *q = m->q;
    return BM_OK;
}

int bm_model_set_engine(bm_model m, int engine)
{
    if (!m) return bm_fail(BM_EINVAL, "bm_model_set_engine: NULL model");
    if (engine != BM_ENGINE_SIMT && engine != BM_ENGINE_AUTO && engine != BM_ENGINE_MMA &&
        engine != BM_ENGINE_MMA_PAIR && engine != BM_ENGINE_MMA_PAIR2)
        return bm_fail(BM_EINVAL, "bm_model_set_engine: unknown engine %d", engine);
    m->engine = engine;
    return BM_OK;
}

int bm_model_set_sampler(bm_model m, int sampler)
{
    if (!m) return bm_fail(BM_EINVAL, "bm_model_set_sampler: NULL model");
    if (sampler != BM_SAMPLER_GIBBS && sampler != BM_SAMPLER_METROPOLIS)
        return bm_fail(BM_EINVAL, "bm_model_set_sampler: unknown sampler %d", sampler);
    m->sampler = sampler;
    return BM_OK;
}

int bm_model_sweep_engine(bm_model m, int M, int *engine_out)
{
    if (!m || !engine_out || M < 1) return bm_fail(BM_EINVAL, "bm_model_sweep_engine: bad argument");
    const int form = bm_sweep_form(m, M);
    *engine_out = form == 3   ? BM_ENGINE_MMA_PAIR2
                  : form == 2 ? BM_ENGINE_MMA_PAIR
                  : form == 1 ? BM_ENGINE_MMA
                              : BM_ENGINE_SIMT;
    return BM_OK;
}

static int chains_init(bm_model m, int M, uint64_t seed, uint64_t chain0, const uint8_t *init_or_null, int where,
                       void *stream, bm_chains *out)
{
    if (!out) return bm_fail(BM_EINVAL, "bm_chains_init: out is NULL");
    *out = nullptr;
    if (!m) return bm_fail(BM_EINVAL, "bm_chains_init: NULL model");
    if (M < 1) return bm_fail(BM_EINVAL, "bm_chains_init: M=%d < 1", M);
    if (init_or_null && !valid_where(where)) return bm_fail(BM_EINVAL, "bm_chains_init: bad where");
    cudaStream_t st = (cudaStream_t)stream;
    bm_chains_s *c = new (std::nothrow) bm_chains_s();
    if (!c) return bm_fail(BM_ENOMEM, "bm_chains_init: host allocation failed");
    c->M = M;
    c->L = m->L;
    c->q = m->q;
    c->device = m->device;
    c->seed = seed;
    c->sweep = 0;
    c->chain0 = chain0;
    const size_t n = (size_t)M * m->L;
    cudaError_t e = cudaMalloc(&c->s, n);
    if (e == cudaSuccess) e = cudaMalloc(&c->derr, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(c->derr, 0, sizeof(int), st);
    if (e != cudaSuccess) {
        cudaFree(c->s);
        cudaFree(c->derr);
        delete c;
        return bm_cuda_fail(e, "cudaMalloc(chains)");
    }
    int rc = BM_OK;
    if (init_or_null) {
        e = cudaMemcpyAsync(c->s, init_or_null, n, copy_kind(where, BM_DEVICE), st);
        if (e != cudaSuccess) rc = bm_cuda_fail(e, "cudaMemcpyAsync(chains init)");
        if (rc == BM_OK) rc = bm_launch_check_symbols(c->s, n, m->q, m->dflags + 1, st);
        int bad = 0;
        if (rc == BM_OK) {
            e = cudaMemcpyAsync(&bad, m->dflags + 1, sizeof(int), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) rc = bm_cuda_fail(e, "check chain symbols");
        }
        if (rc == BM_OK && bad) rc = bm_fail(BM_EINVAL, "bm_chains_init: symbol >= q in init");
    } else {
        rc = bm_launch_chains_init(c->s, M, m->L, m->q, seed, chain0, st);
    }
    if (rc != BM_OK) {
        cudaFree(c->s);
        cudaFree(c->derr);
        delete c;
        return rc;
    }
    *out = c;
    return BM_OK;
}

int bm_chains_init(bm_model m, int M, uint64_t seed, const uint8_t *init_or_null, int where,
                   void *stream, bm_chains *out)
{
    return chains_init(m, M, seed, 0, init_or_null, where, stream, out);
}

int bm_chains_init_shard(bm_model m, int M, uint64_t seed, uint64_t chain0, void *stream, bm_chains *out)
{
    return chains_init(m, M, seed, chain0, nullptr, BM_DEVICE, stream, out);
}

int bm_chains_free(bm_chains c)
{
    if (!c) return BM_OK;
    cudaFree(c->s);
    cudaFree(c->derr);
    if (c->xt) cudaFree(c->xt);
    if (c->ct_ws) cudaFree(c->ct_ws);
    if (c->ct_cnt) cudaFree(c->ct_cnt);
    delete c;
    return BM_OK;
}

int bm_chains_device_status(bm_chains c, void *stream)
{
    if (!c) return bm_fail(BM_EINVAL, "bm_chains_device_status: NULL chains");
    cudaStream_t st = (cudaStream_t)stream;
    int word = 0;
    BM_CK(cudaMemcpyAsync(&word, c->derr, sizeof(int), cudaMemcpyDeviceToHost, st));
    BM_CK(cudaStreamSynchronize(st));
    if (word) {
        BM_CK(cudaMemsetAsync(c->derr, 0, sizeof(int), st));
        return bm_fail(BM_ETIMEOUT, "device wait timed out in a chain-statistics launch (error word 0x%x)", word);
    }
    return BM_OK;
}

int bm_chains_set_stats_engine(bm_chains c, int engine)
{
    if (!c) return bm_fail(BM_EINVAL, "bm_chains_set_stats_engine: NULL chains");
    if (engine < BM_STATS_AUTO || engine > BM_STATS_MMA_FP8)
        return bm_fail(BM_EINVAL, "bm_chains_set_stats_engine: unknown engine %d", engine);
    c->stats_engine = engine;
    return BM_OK;
}

int bm_chains_get(bm_chains c, uint8_t *dst, int where, void *stream)
{
    if (!c || !dst) return bm_fail(BM_EINVAL, "bm_chains_get: NULL argument");
    if (!valid_where(where)) return bm_fail(BM_EINVAL, "bm_chains_get: bad where");
    BM_CK(cudaMemcpyAsync(dst, c->s, (size_t)c->M * c->L, copy_kind(BM_DEVICE, where),
                          (cudaStream_t)stream));
    return BM_OK;
}

int bm_chains_set(bm_chains c, const uint8_t *src, int where, void *stream)
{
    if (!c || !src) return bm_fail(BM_EINVAL, "bm_chains_set: NULL argument");
    if (!valid_where(where)) return bm_fail(BM_EINVAL, "bm_chains_set: bad where");
    BM_CK(cudaMemcpyAsync(c->s, src, (size_t)c->M * c->L, copy_kind(where, BM_DEVICE),
                          (cudaStream_t)stream));
    return BM_OK;
}

int bm_chains_sweep_counter(bm_chains c, uint64_t *sweep)
{
    if (!c || !sweep) return bm_fail(BM_EINVAL, "bm_chains_sweep_counter: NULL argument");
    *sweep = c->sweep;
    return BM_OK;
}

int bm_chains_set_sweep_counter(bm_chains c, uint64_t sweep)
{
    if (!c) return bm_fail(BM_EINVAL, "bm_chains_set_sweep_counter: NULL chains");
    c->sweep = sweep;
    return BM_OK;
}

int bm_chains_shape(bm_chains c, int *M, int *L)
{
    if (!c) return bm_fail(BM_EINVAL, "bm_chains_shape: NULL chains");
    if (M) *M = c->M;
    if (L) *L = c->L;
    return BM_OK;
}

int bm_gibbs_sweep(bm_model m, bm_chains c, int nsweeps, float beta, void *stream)
{
    if (!m || !c) return bm_fail(BM_EINVAL, "bm_gibbs_sweep: NULL handle");
    if (c->L != m->L || c->q != m->q)
        return bm_fail(BM_EINVAL, "bm_gibbs_sweep: chains (L=%d,q=%d) do not match model (L=%d,q=%d)",
                       c->L, c->q, m->L, m->q);
    if (nsweeps < 0) return bm_fail(BM_EINVAL, "bm_gibbs_sweep: nsweeps=%d < 0", nsweeps);
    if (!isfinite(beta)) return bm_fail(BM_EINVAL, "bm_gibbs_sweep: beta not finite");
    return bm_sweep_run(m, c, nsweeps, beta, (cudaStream_t)stream);
}

}  // extern "C"

// AUTO: do the tensor-core forms beat the CUDA-core gather for this shape?
// Measured on an L x q x M grid (L 48-400, q 4-21, M 1000-20000): the
// tensor-core forms redraw the sites of a block one after another, which
// puts a floor of a few microseconds per site under a sweep, so short
// sequences with few chains go to the gather.  Rule: tensor cores from
// L = 120 (and M >= 512), and for alphabets of 10 or more symbols also from
// L = 48 once M * L >= 3e5.
static bool tensor_beats_gather(int L, int q, int M)
{
    if (L >= 120) return M >= 512;
    return q >= 10 && L >= 48 && (double)M * L >= 3e5;
}

int bm_sweep_form(const bm_model_s *m, int M)
{
    if (m->engine == BM_ENGINE_MMA_PAIR2) return 3;
    if (m->engine == BM_ENGINE_MMA_PAIR) return 2;
    if (m->engine == BM_ENGINE_MMA) {
        // the one-CTA form draws Gibbs updates only; Metropolis sweeps run
        // on the two-CTA form (or the CUDA cores where that does not fit)
        if (m->sampler == BM_SAMPLER_METROPOLIS) return bm_gibbs_pair_waves(m, M) > 0 ? 2 : 0;
        return 1;
    }
    if (m->engine != BM_ENGINE_AUTO) return 0;
    if (!tensor_beats_gather(m->L, m->q, M)) return 0;
    // Among the tensor-core forms (same grid; the one-CTA form was never the
    // fastest): the two-CTA engine (form 2) and the paired-tensor-core form
    // (form 3) trade places with the cluster count.
    const int w3 = bm_gibbs_paired_waves(m, M), w2 = bm_gibbs_pair_waves(m, M);
    if (w3 == 0)
        return w2 > 0 ? 2 : (bm_gibbs_mma_chains_per_cta(m, M) > 0 && m->sampler == BM_SAMPLER_GIBBS ? 1 : 0);
    if (w2 == 0) return 3;
    if (bm_gibbs_pair_tm(m)) {
        // form 2 runs its tensor-memory operand form here, 128 chains per
        // cluster: the paired form wins where it fits one wave and form 2
        // does not, or where it spreads the chains at most 32 per cluster
        if (w3 == 1 && w2 > 1) return 3;
        return bm_gibbs_paired_chains_per_cluster(m, M) <= 32 ? 3 : 2;
    }
    // both with shared-memory operands: halving each SM's one-hot work pays
    // while the pair's MMAs are short (L q^2 below ~90,000: q = 21 up to
    // L ~ 200, q = 12 up to L ~ 600)
    return (long long)m->L * m->q * m->q < 90000 ? 3 : 2;
}

int bm_gather_prepare(bm_model_s *m, cudaStream_t st)
{
    if (m->jg_current) return BM_OK;
    const int rc = bm_launch_build_gather(m->J, m->Jg, m->L, m->q, st);
    if (rc == BM_OK) m->jg_current = true;
    return rc;
}

int bm_sweep_run(bm_model_s *m, bm_chains_s *c, int nsweeps, float beta, cudaStream_t st)
{
    const int form = bm_sweep_form(m, c->M);
    if (form == 0) {  // the CUDA-core sweep reads the gather layout
        const int rc = bm_gather_prepare(m, st);
        if (rc != BM_OK) return rc;
    }
    for (int done = 0; done < nsweeps;) {
        const int k = nsweeps - done < kMaxSweepsPerLaunch ? nsweeps - done : kMaxSweepsPerLaunch;
        const int rc = form == 3   ? bm_launch_gibbs_paired(m, c, k, beta, st)
                       : form == 2 ? bm_launch_gibbs_pair(m, c, k, beta, st)
                       : form == 1 ? bm_launch_gibbs_mma(m, c, k, beta, st)
                                   : bm_launch_gibbs_simt(m, c, k, beta, st);
        if (rc != BM_OK) return rc;
        c->sweep += (uint64_t)k;
        done += k;
    }
    return BM_OK;
}

extern "C" {

int bm_chain_stats(bm_chains c, int32_t *counts_dev, void *stream)
{
    if (!c || !counts_dev) return bm_fail(BM_EINVAL, "bm_chain_stats: NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    const bool mma_ok = c->M < (1 << 24);  // FP32 accumulation is exact below 2^24
    switch (c->stats_engine) {
    case BM_STATS_MMA_BF16:
        if (mma_ok) return bm_launch_chain_stats_mma(c->s, c->M, c->L, c->q, counts_dev, 2, c->derr, st);
        break;
    case BM_STATS_AUTO:  // the TMA-fed FP8 product is the faster form when its FP32 counts are exact
    case BM_STATS_MMA_FP8:
        if (mma_ok) return bm_launch_chain_stats_tc(c, counts_dev, st);
        break;
    default:  // BM_STATS_SIMT
        break;
    }
    return bm_launch_chain_stats(c->s, c->M, c->L, c->q, counts_dev, st);
}

int bm_seq_weights(const uint8_t *msa_dev, int N, int L, double seqid, float *w_dev,
                   double *meff_host, void *stream)
{
    if (!msa_dev || !w_dev) return bm_fail(BM_EINVAL, "bm_seq_weights: NULL argument");
    if (N < 1 || L < 1 || L > 4096) return bm_fail(BM_EINVAL, "bm_seq_weights: bad N=%d or L=%d", N, L);
    if (!(seqid > 0.0 && seqid <= 1.0)) return bm_fail(BM_EINVAL, "bm_seq_weights: seqid out of (0,1]");
    cudaStream_t st = (cudaStream_t)stream;
    const int thr = (int)ceil(seqid * L - 1e-9);
    void *scratch = nullptr;
    const size_t cnt_bytes = ((size_t)N * sizeof(int) + 255) & ~(size_t)255;
    const size_t bytes = 256 + cnt_bytes + bm_seq_weights_planes_bytes(N, L);
    BM_CK(cudaMallocAsync(&scratch, bytes, st));
    double *meff_dev = (double *)scratch;
    int *cnt = (int *)((char *)scratch + 256);
    uint32_t *planes = (uint32_t *)((char *)scratch + 256 + cnt_bytes);
    int rc = bm_launch_seq_weights_bs(msa_dev, N, L, thr, w_dev, cnt, planes, meff_dev, st);
    double meff = 0.0;
    if (rc == BM_OK && meff_host) {
        cudaError_t e = cudaMemcpyAsync(&meff, meff_dev, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = bm_cuda_fail(e, "bm_seq_weights: read M_eff");
        else *meff_host = meff;
    }
    cudaFreeAsync(scratch, st);
    return rc;
}

int bm_data_stats(const uint8_t *msa_dev, const float *w_or_null, int N, int L, int q,
                  double pseudocount, float *fi_dev, float *fij_dev, void *stream)
{
    if (!msa_dev || !fi_dev || !fij_dev) return bm_fail(BM_EINVAL, "bm_data_stats: NULL argument");
    if (N < 1 || L < 1 || L > 4096 || q < 1 || q > 32)
        return bm_fail(BM_EINVAL, "bm_data_stats: bad N=%d, L=%d or q=%d", N, L, q);
    if (!(pseudocount <= 1.0)) return bm_fail(BM_EINVAL, "bm_data_stats: pseudocount > 1 or NaN");
    cudaStream_t st = (cudaStream_t)stream;
    double *dtmp = nullptr;
    BM_CK(cudaMallocAsync((void **)&dtmp, 4 * sizeof(double), st));
    double h3[3] = {(double)N, 1.0, 1.0};
    int rc = bm_launch_check_symbols(msa_dev, (size_t)N * L, q, (int *)(dtmp + 3), st);
    int bad = 0;
    if (rc == BM_OK && w_or_null) rc = bm_launch_weight_sum(w_or_null, N, dtmp, st);
    if (rc == BM_OK) {
        cudaError_t e = cudaSuccess;
        if (w_or_null) e = cudaMemcpyAsync(h3, dtmp, 3 * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, dtmp + 3, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = bm_cuda_fail(e, "bm_data_stats: checks");
    }
    cudaFreeAsync(dtmp, st);
    if (rc != BM_OK) return rc;
    if (bad) return bm_fail(BM_EINVAL, "bm_data_stats: symbol >= q in MSA");
    const double meff = h3[0];
    if (!isfinite(h3[1]) || h3[2] < 0.0) return bm_fail(BM_EINVAL, "bm_data_stats: weights must be finite and >= 0");
    if (!(meff > 0.0) || meff >= 4194304.0)
        return bm_fail(BM_EINVAL, "bm_data_stats: sum of weights %.6g outside (0, 2^22)", meff);
    const double alpha = pseudocount < 0.0 ? 1.0 / meff : pseudocount;
    return bm_launch_data_stats(msa_dev, w_or_null, N, L, q, alpha, 40, meff, fi_dev, fij_dev,
                                nullptr, st);
}

int bm_update(bm_model m, const float *fi_data, const float *fij_data, const int32_t *counts,
              int M, float lr, double target, double *pearson_out, int *applied_out, void *stream)
{
    if (!m || !fi_data || !fij_data || !counts) return bm_fail(BM_EINVAL, "bm_update: NULL argument");
    if (M < 1) return bm_fail(BM_EINVAL, "bm_update: M=%d < 1", M);
    if (!isfinite(lr)) return bm_fail(BM_EINVAL, "bm_update: lr not finite");
    cudaStream_t st = (cudaStream_t)stream;
    const int nparts = bm_update_num_partials(m->L, m->q);
    double *partials = m->dred;
    double *moments = m->dred + (size_t)nparts * 5;
    const int want = pearson_out != nullptr;
    int rc = bm_launch_update(m, fi_data, fij_data, counts, M, lr, want, partials, nparts, moments, st);
    if (rc != BM_OK) return rc;
    bool apply = true;
    if (want) {
        double mo[5];
        int word = 0;
        BM_CK(cudaMemcpyAsync(mo, moments, sizeof mo, cudaMemcpyDeviceToHost, st));
        BM_CK(cudaMemcpyAsync(&word, m->dflags + 3, sizeof(int), cudaMemcpyDeviceToHost, st));
        BM_CK(cudaStreamSynchronize(st));
        if (word) {
            BM_CK(cudaMemsetAsync(m->dflags + 3, 0, sizeof(int), st));
            return bm_fail(BM_ETIMEOUT, "bm_update: an earlier Gibbs launch timed out (error word 0x%x)", word);
        }
        const double n = (double)m->L * (m->L - 1) / 2 * m->q * m->q;
        const double cov = n * mo[4] - mo[0] * mo[1];
        const double vx = n * mo[2] - mo[0] * mo[0], vy = n * mo[3] - mo[1] * mo[1];
        const double rho = (vx > 0.0 && vy > 0.0) ? cov / sqrt(vx * vy) : NAN;
        *pearson_out = rho;
        apply = !(rho >= target);
    }
    if (apply) {
        float *t = m->h; m->h = m->h_back; m->h_back = t;
        t = m->J; m->J = m->J_back; m->J_back = t;
        m->mma_current = false;
        m->bf_current = false;
        m->corr_current = false;
        m->jg_current = false;  // rebuilt by the next reader of the gather layout
    }
    if (applied_out) *applied_out = apply ? 1 : 0;
    return BM_OK;
}

int bm_energy_score(bm_model m, const uint8_t *seqs_dev, int n, float *E_dev, void *stream)
{
    if (!m || (n > 0 && (!seqs_dev || !E_dev))) return bm_fail(BM_EINVAL, "bm_energy_score: NULL argument");
    if (n < 0) return bm_fail(BM_EINVAL, "bm_energy_score: n=%d < 0", n);
    const int rc = bm_gather_prepare(m, (cudaStream_t)stream);
    if (rc != BM_OK) return rc;
    return bm_launch_energy(m, seqs_dev, n, E_dev, m->dflags + 4, (cudaStream_t)stream);
}

int bm_fields(bm_model m, const uint8_t *seqs_dev, int n, float *H_dev, int form, void *stream)
{
    if (!m || (n > 0 && (!seqs_dev || !H_dev))) return bm_fail(BM_EINVAL, "bm_fields: NULL argument");
    if (n < 0) return bm_fail(BM_EINVAL, "bm_fields: n=%d < 0", n);
    cudaStream_t st = (cudaStream_t)stream;
    switch (form) {
    case BM_FIELDS_FP32: {
        const int rc = bm_gather_prepare(m, st);
        return rc != BM_OK ? rc : bm_launch_fields_simt(m, seqs_dev, n, H_dev, st);
    }
    case BM_FIELDS_FP16X2: return bm_launch_fields_tc(m, seqs_dev, n, H_dev, 0, st);
    case BM_FIELDS_BF16X2: return bm_launch_fields_tc(m, seqs_dev, n, H_dev, 1, st);
    default: return bm_fail(BM_EINVAL, "bm_fields: unknown form %d", form);
    }
}

int bm_mutant_scan(bm_model m, const uint8_t *wt, int where, float *dE_dev, void *stream)
{
    if (!m || !wt || !dE_dev) return bm_fail(BM_EINVAL, "bm_mutant_scan: NULL argument");
    if (!valid_where(where)) return bm_fail(BM_EINVAL, "bm_mutant_scan: bad where");
    cudaStream_t st = (cudaStream_t)stream;
    if (where == BM_HOST) {
        for (int i = 0; i < m->L; ++i)
            if (wt[i] >= m->q) return bm_fail(BM_EINVAL, "bm_mutant_scan: wt[%d]=%d >= q", i, wt[i]);
    }
    uint8_t *dwt = nullptr;
    BM_CK(cudaMallocAsync((void **)&dwt, (size_t)m->L, st));
    int rc = BM_OK;
    cudaError_t e = cudaMemcpyAsync(dwt, wt, (size_t)m->L, copy_kind(where, BM_DEVICE), st);
    if (e != cudaSuccess) rc = bm_cuda_fail(e, "bm_mutant_scan: copy wt");
    if (rc == BM_OK && where == BM_DEVICE) {
        int bad = 0;
        rc = bm_launch_check_symbols(dwt, (size_t)m->L, m->q, m->dflags + 2, st);
        if (rc == BM_OK) {
            e = cudaMemcpyAsync(&bad, m->dflags + 2, sizeof(int), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) rc = bm_cuda_fail(e, "bm_mutant_scan: check wt");
            else if (bad) rc = bm_fail(BM_EINVAL, "bm_mutant_scan: wt symbol >= q");
        }
    }
    if (rc == BM_OK) rc = bm_launch_mutant_scan(m->h, m->J, m->L, m->q, dwt, dE_dev, st);
    cudaFreeAsync(dwt, st);
    return rc;
}

}  // extern "C"
