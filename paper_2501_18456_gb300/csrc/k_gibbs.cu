// Persistent-chain Gibbs sampling on CUDA cores (FP32), and chain
// initialisation.
//
// Method (adabmDCA 2.0, Sec. 2.1 "Monte Carlo estimation of the gradient";
// a sweep proposes every site once, Sec. 3.3): for each chain and each site
// i = 0..L-1 in order, the local field H_i(a) = h_i(a) + sum_{j != i}
// J_ij(a, s_j) (Eq. 1 with all other sites fixed) is formed from the
// current state and s_i is redrawn from p(a) ~ exp(beta H_i(a)).
//
// Data path.  The model keeps a gather layout Jg[i][j][b][a] = J_ij(a,b)
// with each (i,j) block padded to bs floats (a multiple of 4, so every block
// starts on a 16-byte boundary): the data needed to update site i is the
// contiguous slab Jg[i][0..L).  One CTA per SM owns ~M/#SM chains and walks
// the sites in lock-step; a producer warp streams the slab of the current
// site through a ring of shared-memory stages with cp.async.bulk (one bulk
// copy of JC blocks per stage, completion counted on an mbarrier), and the
// consumer warps gather from shared memory: a group of GW lanes (GW = q
// rounded up to a power of two) owns R chains, lane a accumulates H_i(a),
// reading row Jg[i][j][s_j][.] of the staged slab.  J_ii = 0 is enforced at
// load, so the j = i term adds an exact zero.  All nsweeps sweeps run in one
// launch: chains are independent and need no grid-wide synchronisation.
//
// Every mbarrier wait is bounded by %globaltimer (2 s).  A wait that runs
// out sets an abort flag in shared memory and bit 0 of the model's device
// error word; all warps then leave their loops, the producer waits (again
// bounded) for the copies it issued, chain states are left unchanged and
// the host reports BM_ETIMEOUT at its next synchronising call.
#include "bm_internal.cuh"

#include <algorithm>
#include <new>
#include <vector>

namespace {

__global__ void k_chains_init(uint8_t *__restrict__ s, int M, int L, int q, uint64_t seed, uint64_t chain0)
{
    const size_t n = (size_t)M * L;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (size_t)gridDim.x * blockDim.x) {
        const uint64_t m = t / (size_t)L, i = t % (size_t)L;
        const uint64_t r = bm_u24(seed, chain0 + m, 0, i, 1);
        s[t] = (uint8_t)((r * (uint64_t)q) >> 24);
    }
}

// Jg[i][j][b][a] = J_ij(a,b) = J[j][i][b][a] (symmetry): block (i,j) of the
// gather layout is a plain copy of block (j,i) of the natural layout.
__global__ void k_build_gather(const float *__restrict__ J, float *__restrict__ Jg, int L, int q,
                               int bs)
{
    const int qq = q * q;
    const size_t nblk = (size_t)L * L;
    for (size_t blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
        const size_t i = blk / L, j = blk % L;
        const float *src = J + (j * L + i) * (size_t)qq;
        float *dst = Jg + blk * (size_t)bs;
        for (int e = threadIdx.x; e < bs; e += blockDim.x) dst[e] = e < qq ? src[e] : 0.0f;
    }
}

// ---------------------------------------------------------------------------
// mbarrier / bulk-copy helpers (inline PTX, sm_90+ forms valid on sm_103a)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s

// Bounded wait: true when the phase with `parity` has completed; false after
// an abort (raised here on timeout, or earlier by another warp).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag,
                                          int *err, uint64_t limit_ns = kWaitLimitNs)
{
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (*abort_flag) return false;
        if (globaltimer_ns() - t0 > limit_ns) {
            *abort_flag = 1;
            atomicOr(err, 1);
            return false;
        }
    }
}

// Shared-memory load through a 32-bit shared-window address.  Volatile so
// that it stays between the stage's mbarrier wait and the release of the
// stage (both volatile asm with memory clobbers).
__device__ __forceinline__ float lds_f32(uint32_t addr)
{
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr));
    return v;
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

struct GibbsArgs {
    const float *h;
    const float *Jg;
    uint8_t *states;
    int *err;
    uint64_t seed, sweep0, chain0;  // chain0: global index of chain 0 (Philox counter)
    float beta;
    int M, L, q, Lp, bs, jc, nch, ns, cpc, nsweeps;
    int sampler;  // BM_SAMPLER_GIBBS or BM_SAMPLER_METROPOLIS
};

// One CTA of a batched launch: the model and chains it works on (h, Jg,
// states, err, seed, sweep0, M, L, Lp, nch differ per model; the rest is
// the launch's common shape) and the index of its first chain.
struct BatchItem {
    GibbsArgs a;
    long long first;  // first chain of the tile (index into the model's chains)
};

// Shared memory: [ns stages of jc*bs floats][cpc x Lp u32 row offsets]
// [2*ns mbarriers][abort flag].  The row offset of chain c at site j is
// the byte offset, inside a stage, of row (j mod jc, s_j):
//     os[c][j] = ((j mod jc) * bs + s_j * q) * 4,
// so the gather of a staged element is a single shared load at
// stage base + lane column + os (the chain state is recovered from it at
// the end of the launch).
//
// GW: lanes per chain group (power of two >= q); R: chains per group;
// JCC: compile-time chunk length for fully unrolled full chunks (0: use the
// runtime loop for every chunk).  blockDim = (consumer warps + 1) * 32; the
// last warp is the producer.
template <int GW, int R, int JCC, bool BATCH>
__global__ void __launch_bounds__(1024, 1) k_gibbs_staged(const GibbsArgs p0, const BatchItem *__restrict__ items)
{
    constexpr int G = 32 / GW;
    // batched launch: this CTA's model and first chain come from the work list
    const GibbsArgs p = BATCH ? items[blockIdx.x].a : p0;
    const size_t cta0 = BATCH ? (size_t)items[blockIdx.x].first : (size_t)blockIdx.x * p0.cpc;
    extern __shared__ __align__(128) unsigned char smem[];
    const int nwc = (blockDim.x >> 5) - 1;  // consumer warps
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t stage_bytes = (uint32_t)p.jc * (uint32_t)p.bs * 4u;
    uint32_t *os = reinterpret_cast<uint32_t *>(smem + (size_t)p.ns * stage_bytes);
    uint64_t *bars = reinterpret_cast<uint64_t *>(os + (size_t)p.cpc * p.Lp);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(bars + 2 * p.ns);
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + p.ns);
    const uint32_t rowb = (uint32_t)p.q * 4u, jstep = (uint32_t)p.bs * 4u;

    if (threadIdx.x == 0) {
        for (int s = 0; s < p.ns; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, (uint32_t)nwc);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int k = threadIdx.x; k < p.cpc * p.Lp; k += blockDim.x) {
        const int c = k / p.Lp, x = k - c * p.Lp;
        const size_t m = cta0 + c;
        const uint32_t sv = (m < (size_t)p.M && x < p.L) ? p.states[m * p.L + x] : 0u;
        os[k] = (uint32_t)(x % p.jc) * jstep + sv * rowb;
    }
    __syncthreads();

    const long long total = (long long)p.nsweeps * p.L * p.nch;
    if (warp == nwc) {
        // ------------------------------------------------------- producer
        if (lane != 0) return;
        long long issued = 0;
        for (long long t = 0; t < total; ++t) {
            const int s = (int)(t % p.ns);
            const long long use = t / p.ns;
            if (use > 0 && !mbar_wait(empty0 + 8 * s, (uint32_t)((use - 1) & 1), abort_flag, p.err)) break;
            const long long u = t / p.nch;
            const int c = (int)(t - u * p.nch);
            const int i = (int)(u % p.L);
            const int j0 = c * p.jc;
            const int nj = min(p.jc, p.L - j0);
            const uint32_t bytes = (uint32_t)nj * jstep;
            mbar_arrive_expect_tx(full0 + 8 * s, bytes);
            bulk_g2s(smem_u32(smem + (size_t)s * stage_bytes), p.Jg + ((size_t)i * p.L + j0) * p.bs,
                     bytes, full0 + 8 * s);
            ++issued;
        }
        if (*abort_flag) {
            // Let every copy this thread issued land before the CTA can exit.
            volatile int no_abort = 0;
            for (long long t = issued > p.ns ? issued - p.ns : 0; t < issued; ++t)
                mbar_wait(full0 + 8 * (int)(t % p.ns), (uint32_t)((t / p.ns) & 1), &no_abort, p.err,
                          kWaitLimitNs / 4);
        }
        return;
    }

    // ----------------------------------------------------------- consumers
    const int g = lane / GW, a = lane % GW;
    const int slot0 = (warp * G + g) * R;
    uint32_t *og = os + (size_t)slot0 * p.Lp;
    const int q = p.q;
    const int aa = a < q ? a : q - 1;  // idle lanes mirror column q-1
    const unsigned gmask = (GW == 32) ? 0xffffffffu : (((1u << GW) - 1u) << (g * GW));
    bool ok = true;
    long long t = 0;
    for (int sw = 0; sw < p.nsweeps && ok; ++sw) {
        const uint64_t sweep = p.sweep0 + (uint64_t)sw;
        for (int i = 0; i < p.L && ok; ++i) {
            float acc[R];
            const float hv = p.h[(size_t)i * q + aa];
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] = hv;
            for (int c = 0; c < p.nch; ++c, ++t) {
                const int s = (int)(t % p.ns);
                if (!mbar_wait(full0 + 8 * s, (uint32_t)((t / p.ns) & 1), abort_flag, p.err)) {
                    ok = false;
                    break;
                }
                const uint32_t lb = smem_u32(smem) + (uint32_t)s * stage_bytes + (uint32_t)aa * 4u;
                const int j0 = c * p.jc;
                const int nj = min(p.jc, p.L - j0);
                if (JCC > 0 && nj == JCC) {
#pragma unroll
                    for (int jj = 0; jj < JCC; jj += 4) {
                        uint4 o[R];
#pragma unroll
                        for (int r = 0; r < R; ++r)
                            o[r] = *reinterpret_cast<const uint4 *>(og + r * p.Lp + j0 + jj);
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            acc[r] += lds_f32(lb + o[r].x);
                            acc[r] += lds_f32(lb + o[r].y);
                            acc[r] += lds_f32(lb + o[r].z);
                            acc[r] += lds_f32(lb + o[r].w);
                        }
                    }
                } else {
                    for (int jj = 0; jj < nj; ++jj)
#pragma unroll
                        for (int r = 0; r < R; ++r)
                            acc[r] += lds_f32(lb + og[r * p.Lp + j0 + jj]);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(empty0 + 8 * s);
            }
            if (!ok) break;
            const uint32_t ibase = (uint32_t)(i % p.jc) * jstep;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const uint64_t m = p.chain0 + cta0 + slot0 + r;  // global chain index
                if (p.sampler == BM_SAMPLER_METROPOLIS) {
                    // one Metropolis-Hastings step from the current symbol: the
                    // lanes of the proposed and current symbols hold their fields
                    const int cur = (int)((og[r * p.Lp + i] - ibase) / rowb);
                    const uint32_t w = bm_mh_word(p.seed, m, sweep, (uint64_t)i, q);
                    const int prop = (int)(w >> 24) + ((int)(w >> 24) >= cur ? 1 : 0);
                    const float l2e = p.beta * 1.4426950408889634f;
                    const float hp = __shfl_sync(0xffffffffu, acc[r], g * GW + min(prop, q - 1)) * l2e;
                    const float hc = __shfl_sync(0xffffffffu, acc[r], g * GW + cur) * l2e;
                    const int pick = (q > 1 && bm_mh_accept(hp, hc, w)) ? prop : cur;
                    if (a == 0) og[r * p.Lp + i] = ibase + (uint32_t)pick * rowb;
                    continue;
                }
                const float e = (a < q) ? p.beta * acc[r] : -INFINITY;
                const float mx = group_max<GW>(e);
                const float w = (a < q) ? expf(e - mx) : 0.0f;
                const float S = group_inclusive_scan<GW>(w, a);
                const float tot = __shfl_sync(0xffffffffu, S, q - 1, GW);
                const uint32_t r24 = bm_u24(p.seed, m, sweep, (uint64_t)i, 0);
                const float thr = ((float)r24 * 5.9604644775390625e-8f) * tot;  // u * S_total
                const unsigned bal = __ballot_sync(0xffffffffu, (a < q) && (thr < S)) & gmask;
                const int pick = bal ? (__ffs(bal) - 1 - g * GW) : (q - 1);
                if (a == 0) og[r * p.Lp + i] = ibase + (uint32_t)pick * rowb;
            }
            __syncwarp();
        }
    }
    if (!ok) return;  // aborted: leave the chains as they were
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const size_t m = cta0 + slot0 + r;
        if (m < (size_t)p.M)
            for (int k = a; k < p.L; k += GW)
                p.states[m * p.L + k] =
                    (uint8_t)((og[r * p.Lp + k] - (uint32_t)(k % p.jc) * jstep) / rowb);
    }
}

struct Shape {
    int GW, R, cpc, warps, jc, ns, grid, jcc;
    size_t smem;
};

constexpr size_t kSmemBudget = 224 * 1024;
constexpr size_t kStageTarget = 28 * 1024;

Shape pick_shape(const bm_model_s *m, int M)
{
    Shape s{};
    const int q = m->q, L = m->L;
    s.GW = q <= 4 ? 4 : q <= 8 ? 8 : q <= 16 ? 16 : 32;
    const int G = 32 / s.GW;
    const size_t row = (size_t)m->bs * 4;  // bytes per (i,j) block
    int jc = (int)(kStageTarget / row);
    jc = std::max(4, std::min(64, jc & ~3));
    s.jc = std::min(jc, (L + 3) & ~3);
    const size_t stage = (size_t)s.jc * row;
    const int Lp = (L + 15) & ~15;
    const int nsm = m->num_sms > 0 ? m->num_sms : 1;
    int cpc = (M + nsm - 1) / nsm;
    // at least 2 stages; up to 4 while chains' offsets still fit
    const size_t fixed = 64;
    const int cap_smem = (int)((kSmemBudget - 2 * stage - fixed) / ((size_t)Lp * 4));
    cpc = std::max(1, std::min(cpc, cap_smem));
    cpc = std::min(cpc, 31 * G * 4);
    int R = (cpc + 31 * G - 1) / (31 * G);
    R = std::max(1, std::min(4, R));
    int warps = (cpc + G * R - 1) / (G * R);
    warps = std::max(1, std::min(31, warps));
    s.R = R;
    s.warps = warps;
    s.cpc = warps * G * R;
    const size_t osb = (size_t)s.cpc * Lp * 4;
    s.ns = (int)std::min<size_t>(4, (kSmemBudget - osb - fixed) / stage);
    s.ns = std::max(2, s.ns);
    s.grid = (M + s.cpc - 1) / s.cpc;
    s.smem = (size_t)s.ns * stage + osb + 2 * s.ns * 8 + 16;
    s.jcc = (s.GW == 32 && s.jc == 16) ? 16 : (s.GW == 8 && s.jc == 64) ? 64 : 0;
    return s;
}

// attr_only: set the kernel's shared-memory limit and launch nothing (done
// before a stream capture).
template <int GW, int R, int JCC>
int launch_staged(const GibbsArgs &a, const Shape &s, cudaStream_t st, const BatchItem *items = nullptr,
                  bool attr_only = false)
{
    if (items) {
        auto kern = k_gibbs_staged<GW, R, JCC, true>;
        if (attr_only) {
            BM_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.smem));
            return BM_OK;
        }
        kern<<<s.grid, (s.warps + 1) * 32, s.smem, st>>>(a, items);
    } else {
        auto kern = k_gibbs_staged<GW, R, JCC, false>;
        BM_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.smem));
        kern<<<s.grid, (s.warps + 1) * 32, s.smem, st>>>(a, nullptr);
    }
    BM_CK_LAUNCH("k_gibbs_staged");
    return BM_OK;
}

template <int GW, int JCC>
int dispatch_r(const GibbsArgs &a, const Shape &s, cudaStream_t st, const BatchItem *items = nullptr,
               bool attr_only = false)
{
    switch (s.R) {
    case 1: return launch_staged<GW, 1, JCC>(a, s, st, items, attr_only);
    case 2: return launch_staged<GW, 2, JCC>(a, s, st, items, attr_only);
    case 3: return launch_staged<GW, 3, JCC>(a, s, st, items, attr_only);
    default: return launch_staged<GW, 4, JCC>(a, s, st, items, attr_only);
    }
}

int dispatch_shape(const GibbsArgs &a, const Shape &s, cudaStream_t st, const BatchItem *items,
                   bool attr_only = false)
{
    if (s.jcc == 16) return dispatch_r<32, 16>(a, s, st, items, attr_only);
    if (s.jcc == 64) return dispatch_r<8, 64>(a, s, st, items, attr_only);
    switch (s.GW) {
    case 4: return dispatch_r<4, 0>(a, s, st, items, attr_only);
    case 8: return dispatch_r<8, 0>(a, s, st, items, attr_only);
    case 16: return dispatch_r<16, 0>(a, s, st, items, attr_only);
    default: return dispatch_r<32, 0>(a, s, st, items, attr_only);
    }
}

}  // namespace

int bm_launch_chains_init(uint8_t *s, int M, int L, int q, uint64_t seed, uint64_t chain0, cudaStream_t st)
{
    const size_t n = (size_t)M * L;
    const int grid = (int)std::min<size_t>((n + 255) / 256, 65535);
    k_chains_init<<<grid, 256, 0, st>>>(s, M, L, q, seed, chain0);
    BM_CK_LAUNCH("k_chains_init");
    return BM_OK;
}

int bm_gather_block_stride(int q) { return (q * q + 3) & ~3; }

int bm_launch_build_gather(const float *J, float *Jg, int L, int q, cudaStream_t st)
{
    const size_t nblk = (size_t)L * L;
    const int grid = (int)std::min<size_t>(nblk, 152 * 32);
    k_build_gather<<<grid, 128, 0, st>>>(J, Jg, L, q, bm_gather_block_stride(q));
    BM_CK_LAUNCH("k_build_gather");
    return BM_OK;
}

int bm_launch_gibbs_simt(const bm_model_s *m, bm_chains_s *c, int nsweeps, float beta,
                         cudaStream_t st)
{
    const Shape s = pick_shape(m, c->M);
    GibbsArgs a;
    a.h = m->h;
    a.Jg = m->Jg;
    a.states = c->s;
    a.err = m->dflags + 3;
    a.seed = c->seed;
    a.chain0 = c->chain0;
    a.sweep0 = c->sweep;
    a.beta = beta;
    a.sampler = m->sampler;
    a.M = c->M;
    a.L = c->L;
    a.q = c->q;
    a.Lp = (c->L + 15) & ~15;
    a.bs = m->bs;
    a.jc = s.jc;
    a.nch = (c->L + s.jc - 1) / s.jc;
    a.ns = s.ns;
    a.cpc = s.cpc;
    a.nsweeps = nsweeps;
    return dispatch_shape(a, s, st, nullptr);
}

// ---------------------------------------------------------------------------
// Batched sweeps of many independent models (same q) in one launch.
//
// The work list holds one entry per CTA: a tile of cpc chains of one model.
// Entries are ordered by decreasing cost (L^2 per chain: the longest models
// first, so the tail of the launch is filled with short tiles).  All entries
// share the launch shape (warp layout, stages, chains per CTA, chunk
// length); shared memory is sized for the longest model.  The list lives in
// device memory and is refreshed from a pinned host copy by the first node
// of a captured CUDA graph, so each call is one graph launch that picks up
// the models' current parameter pointers and sweep counters.
// ---------------------------------------------------------------------------
namespace {

bool batch_shape(int q, int bs, int Lmax, int cpc_target, int ns, int nsm, Shape *out)
{
    Shape s{};
    s.GW = q <= 4 ? 4 : q <= 8 ? 8 : q <= 16 ? 16 : 32;
    const int G = 32 / s.GW;
    const size_t row = (size_t)bs * 4;
    int jc = (int)(kStageTarget / row);
    s.jc = std::max(4, std::min(64, jc & ~3));
    const size_t stage = (size_t)s.jc * row;
    const int Lp = (Lmax + 15) & ~15;
    int R = (cpc_target + 31 * G - 1) / (31 * G);
    R = std::max(1, std::min(4, R));
    int warps = (cpc_target + G * R - 1) / (G * R);
    warps = std::max(1, std::min(31, warps));
    s.R = R;
    s.warps = warps;
    s.cpc = warps * G * R;
    s.ns = ns;
    s.smem = (size_t)ns * stage + (size_t)s.cpc * Lp * 4 + 2 * ns * 8 + 16;
    s.jcc = (s.GW == 32 && s.jc == 16) ? 16 : (s.GW == 8 && s.jc == 64) ? 64 : 0;
    (void)nsm;
    *out = s;
    return s.smem <= kSmemBudget;
}

}  // namespace

struct bm_batch_s {
    std::vector<bm_model_s *> models;
    std::vector<bm_chains_s *> chains;
    int q = 0, bs = 0, Lmax = 0, nsm = 1;
    Shape shape{};
    bool tuned = false;
    int nitems = 0;
    BatchItem *items_dev = nullptr;
    BatchItem *items_host[2] = {nullptr, nullptr};  // pinned, alternating
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    cudaEvent_t used[2] = {nullptr, nullptr};        // last launch that read items_host[k]
    int next = 0;
    std::vector<int> order;                          // model index of each tile, LPT order
    std::vector<long long> first;                    // first chain of each tile
    bm_pair_batch_s *pair = nullptr;                 // tensor-core form (then nothing above is used)
};

namespace {

// Tiles of the batch for chains-per-CTA cpc, longest models first.
void build_tiles(bm_batch_s *b, int cpc)
{
    std::vector<int> idx(b->models.size());
    for (size_t k = 0; k < idx.size(); ++k) idx[k] = (int)k;
    std::stable_sort(idx.begin(), idx.end(), [b](int x, int y) { return b->models[x]->L > b->models[y]->L; });
    b->order.clear();
    b->first.clear();
    for (int k : idx)
        for (long long c0 = 0; c0 < b->chains[k]->M; c0 += cpc) {
            b->order.push_back(k);
            b->first.push_back(c0);
        }
    b->nitems = (int)b->order.size();
}

void fill_items(const bm_batch_s *b, BatchItem *dst, int nsweeps, float beta, uint8_t *const *states_override)
{
    const Shape &s = b->shape;
    for (int t = 0; t < b->nitems; ++t) {
        const int k = b->order[t];
        const bm_model_s *m = b->models[k];
        const bm_chains_s *c = b->chains[k];
        GibbsArgs &a = dst[t].a;
        a.h = m->h;
        a.Jg = m->Jg;
        a.states = states_override ? states_override[k] : c->s;
        a.err = m->dflags + 3;
        a.seed = c->seed;
        a.chain0 = c->chain0;
        a.sweep0 = c->sweep;
        a.beta = beta;
    a.sampler = m->sampler;
        a.M = c->M;
        a.L = c->L;
        a.q = c->q;
        a.Lp = (c->L + 15) & ~15;
        a.bs = m->bs;
        a.jc = s.jc;
        a.nch = (c->L + s.jc - 1) / s.jc;
        a.ns = s.ns;
        a.cpc = s.cpc;
        a.nsweeps = nsweeps;
        dst[t].first = b->first[t];
    }
}

void drop_graphs(bm_batch_s *b)
{
    for (int k = 0; k < 2; ++k) {
        if (b->used[k]) cudaEventSynchronize(b->used[k]);
        if (b->graph[k]) cudaGraphExecDestroy(b->graph[k]);
        b->graph[k] = nullptr;
        cudaFreeHost(b->items_host[k]);
        b->items_host[k] = nullptr;
    }
    cudaFree(b->items_dev);
    b->items_dev = nullptr;
}

// (Re)build the work list, its buffers and the two graphs for the current shape.
int prepare(bm_batch_s *b, cudaStream_t st)
{
    drop_graphs(b);
    build_tiles(b, b->shape.cpc);
    b->shape.grid = b->nitems;
    const size_t bytes = (size_t)b->nitems * sizeof(BatchItem);
    BM_CK(cudaMalloc(&b->items_dev, bytes));
    for (int k = 0; k < 2; ++k) {
        BM_CK(cudaMallocHost(&b->items_host[k], bytes));
        fill_items(b, b->items_host[k], 0, 1.0f, nullptr);
        if (!b->used[k]) BM_CK(cudaEventCreateWithFlags(&b->used[k], cudaEventDisableTiming));
    }
    {
        GibbsArgs dummy{};
        const int rc0 = dispatch_shape(dummy, b->shape, nullptr, b->items_dev, true);
        if (rc0 != BM_OK) return rc0;
    }
    cudaStream_t cap;
    BM_CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    int rc = BM_OK;
    for (int k = 0; k < 2 && rc == BM_OK; ++k) {
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            e = cudaMemcpyAsync(b->items_dev, b->items_host[k], bytes, cudaMemcpyHostToDevice, cap);
            if (e == cudaSuccess) {
                GibbsArgs dummy{};
                rc = dispatch_shape(dummy, b->shape, cap, b->items_dev);
            }
            const cudaError_t e2 = cudaStreamEndCapture(cap, &g);
            if (e == cudaSuccess) e = e2;
        }
        if (e == cudaSuccess && rc == BM_OK) e = cudaGraphInstantiate(&b->graph[k], g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess && rc == BM_OK) rc = bm_cuda_fail(e, "bm_batch: graph capture");
    }
    cudaStreamDestroy(cap);
    (void)st;
    return rc;
}

int launch_graph(bm_batch_s *b, int nsweeps, float beta, cudaStream_t st, uint8_t *const *states_override)
{
    for (bm_model_s *m : b->models) {  // the CUDA-core batch reads each model's gather layout
        const int rc = bm_gather_prepare(m, st);
        if (rc != BM_OK) return rc;
    }
    const int k = b->next;
    b->next ^= 1;
    BM_CK(cudaEventSynchronize(b->used[k]));  // the previous launch that read this host copy has run
    fill_items(b, b->items_host[k], nsweeps, beta, states_override);
    BM_CK(cudaGraphLaunch(b->graph[k], st));
    BM_CK(cudaEventRecord(b->used[k], st));
    return BM_OK;
}

}  // namespace

extern "C" {

int bm_batch_create(const bm_model *models, const bm_chains *chains, int count, bm_batch *out)
{
    if (!out) return bm_fail(BM_EINVAL, "bm_batch_create: out is NULL");
    *out = nullptr;
    if (!models || !chains || count < 1) return bm_fail(BM_EINVAL, "bm_batch_create: empty batch");
    bm_batch_s *b = new (std::nothrow) bm_batch_s();
    if (!b) return bm_fail(BM_ENOMEM, "bm_batch_create: host allocation failed");
    for (int k = 0; k < count; ++k) {
        bm_model_s *m = models[k];
        bm_chains_s *c = chains[k];
        int rc = BM_OK;
        if (!m || !c) rc = bm_fail(BM_EINVAL, "bm_batch_create: NULL handle at %d", k);
        else if (c->L != m->L || c->q != m->q) rc = bm_fail(BM_EINVAL, "bm_batch_create: chains %d do not match model", k);
        else if (k > 0 && m->q != b->q) rc = bm_fail(BM_EINVAL, "bm_batch_create: all models need the same q");
        if (rc != BM_OK) {
            delete b;
            return rc;
        }
        b->models.push_back(m);
        b->chains.push_back(c);
        b->q = m->q;
        b->bs = m->bs;
        b->Lmax = std::max(b->Lmax, m->L);
        b->nsm = m->num_sms > 0 ? m->num_sms : 1;
    }
    // tensor-core form unless a model is held to the CUDA cores (a batch packs
    // every model's tiles into one launch, so the per-model small-problem
    // rule of AUTO does not apply; measured with 64 models, L 50-511,
    // M = 2048: 1.2x to 1.8x the gather's batch for q = 4, 5, 8, 2.9x at 21)
    bool tc = b->q >= 2;
    for (int k = 0; k < count; ++k) tc = tc && b->models[k]->engine != BM_ENGINE_SIMT;
    if (tc && bm_pair_batch_create(b->models.data(), b->chains.data(), count, &b->pair) == BM_OK) {
        *out = b;
        return BM_OK;
    }
    // default shape: the largest chains-per-CTA that fits with 3 stages
    int rc = bm_fail(BM_EINVAL, "bm_batch_create: L=%d does not fit shared memory", b->Lmax);
    for (int cpc : {124, 96, 64, 48, 32, 16, 8}) {
        for (int ns : {3, 2}) {
            Shape s;
            if (batch_shape(b->q, b->bs, b->Lmax, cpc, ns, b->nsm, &s)) {
                b->shape = s;
                rc = BM_OK;
                break;
            }
        }
        if (rc == BM_OK) break;
    }
    if (rc == BM_OK) rc = prepare(b, nullptr);
    if (rc != BM_OK) {
        drop_graphs(b);
        for (auto &e : b->used)
            if (e) cudaEventDestroy(e);
        delete b;
        return rc;
    }
    *out = b;
    return BM_OK;
}

int bm_batch_free(bm_batch b)
{
    if (!b) return BM_OK;
    bm_pair_batch_free(b->pair);
    drop_graphs(b);
    for (auto &e : b->used)
        if (e) cudaEventDestroy(e);
    delete b;
    return BM_OK;
}

int bm_batch_sweep(bm_batch b, int nsweeps, float beta, void *stream)
{
    if (!b) return bm_fail(BM_EINVAL, "bm_batch_sweep: NULL batch");
    if (nsweeps < 0) return bm_fail(BM_EINVAL, "bm_batch_sweep: nsweeps=%d < 0", nsweeps);
    if (!isfinite(beta)) return bm_fail(BM_EINVAL, "bm_batch_sweep: beta not finite");
    if (nsweeps == 0) return BM_OK;
    const int rc = b->pair ? bm_pair_batch_sweep(b->pair, nsweeps, beta, (cudaStream_t)stream, nullptr)
                           : launch_graph(b, nsweeps, beta, (cudaStream_t)stream, nullptr);
    if (rc != BM_OK) return rc;
    for (auto *c : b->chains) c->sweep += (uint64_t)nsweeps;
    return BM_OK;
}

int bm_batch_autotune(bm_batch b, void *stream)
{
    if (!b) return bm_fail(BM_EINVAL, "bm_batch_autotune: NULL batch");
    cudaStream_t st = (cudaStream_t)stream;
    if (b->pair) {
        const int rc = bm_pair_batch_autotune(b->pair, st);
        b->tuned = rc == BM_OK;
        return rc;
    }
    // scratch copies of the states: tuning sweeps must not move the chains
    std::vector<uint8_t *> scratch(b->chains.size(), nullptr);
    int rc = BM_OK;
    for (size_t k = 0; k < b->chains.size() && rc == BM_OK; ++k) {
        const size_t n = (size_t)b->chains[k]->M * b->chains[k]->L;
        cudaError_t e = cudaMalloc(&scratch[k], n);
        if (e == cudaSuccess) e = cudaMemcpyAsync(scratch[k], b->chains[k]->s, n, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) rc = bm_cuda_fail(e, "bm_batch_autotune: scratch");
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (rc == BM_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        rc = bm_fail(BM_ECUDA, "bm_batch_autotune: events");
    Shape best = b->shape;
    float best_ms = 1e30f;
    for (int cpc : {16, 32, 48, 64, 96, 124}) {
        for (int ns : {2, 3, 4}) {
            if (rc != BM_OK) break;
            Shape s;
            if (!batch_shape(b->q, b->bs, b->Lmax, cpc, ns, b->nsm, &s)) continue;
            b->shape = s;
            rc = prepare(b, st);
            if (rc != BM_OK) break;
            rc = launch_graph(b, 1, 1.0f, st, scratch.data());  // warm-up
            if (rc == BM_OK && cudaEventRecord(e0, st) != cudaSuccess) rc = bm_fail(BM_ECUDA, "autotune event");
            for (int r = 0; r < 2 && rc == BM_OK; ++r) rc = launch_graph(b, 1, 1.0f, st, scratch.data());
            if (rc == BM_OK && cudaEventRecord(e1, st) != cudaSuccess) rc = bm_fail(BM_ECUDA, "autotune event");
            float ms = 0.0f;
            if (rc == BM_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                rc = bm_fail(BM_ECUDA, "autotune timing");
            if (rc == BM_OK && ms < best_ms) {
                best_ms = ms;
                best = s;
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(st);
    for (auto *p : scratch) cudaFree(p);
    b->shape = best;
    const int rc2 = prepare(b, st);
    if (rc == BM_OK) rc = rc2;
    b->tuned = rc == BM_OK;
    return rc;
}

int bm_batch_shape(bm_batch b, int *chains_per_cta, int *stages, int *ctas)
{
    if (!b) return bm_fail(BM_EINVAL, "bm_batch_shape: NULL batch");
    if (b->pair) {
        bm_pair_batch_shape(b->pair, chains_per_cta, ctas);
        if (stages) *stages = 2;  // one-hot operand ring of the tensor-core form
        return BM_OK;
    }
    if (chains_per_cta) *chains_per_cta = b->shape.cpc;
    if (stages) *stages = b->shape.ns;
    if (ctas) *ctas = b->nitems;
    return BM_OK;
}

}  // extern "C"
