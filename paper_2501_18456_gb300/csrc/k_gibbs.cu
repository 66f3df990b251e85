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
    uint64_t seed, sweep0;
    float beta;
    int M, L, q, Lp, bs, jc, nch, ns, cpc, nsweeps;
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
template <int GW, int R, int JCC>
__global__ void __launch_bounds__(1024, 1) k_gibbs_staged(const GibbsArgs p)
{
    constexpr int G = 32 / GW;
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
    const size_t cta0 = (size_t)blockIdx.x * p.cpc;
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
                const float e = (a < q) ? p.beta * acc[r] : -INFINITY;
                const float mx = group_max<GW>(e);
                const float w = (a < q) ? expf(e - mx) : 0.0f;
                const float S = group_inclusive_scan<GW>(w, a);
                const float tot = __shfl_sync(0xffffffffu, S, q - 1, GW);
                const uint64_t m = cta0 + slot0 + r;
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

template <int GW, int R, int JCC>
int launch_staged(const GibbsArgs &a, const Shape &s, cudaStream_t st)
{
    auto kern = k_gibbs_staged<GW, R, JCC>;
    BM_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.smem));
    kern<<<s.grid, (s.warps + 1) * 32, s.smem, st>>>(a);
    BM_CK_LAUNCH("k_gibbs_staged");
    return BM_OK;
}

template <int GW, int JCC>
int dispatch_r(const GibbsArgs &a, const Shape &s, cudaStream_t st)
{
    switch (s.R) {
    case 1: return launch_staged<GW, 1, JCC>(a, s, st);
    case 2: return launch_staged<GW, 2, JCC>(a, s, st);
    case 3: return launch_staged<GW, 3, JCC>(a, s, st);
    default: return launch_staged<GW, 4, JCC>(a, s, st);
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
    a.sweep0 = c->sweep;
    a.beta = beta;
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
    if (s.jcc == 16) return dispatch_r<32, 16>(a, s, st);
    if (s.jcc == 64) return dispatch_r<8, 64>(a, s, st);
    switch (s.GW) {
    case 4: return dispatch_r<4, 0>(a, s, st);
    case 8: return dispatch_r<8, 0>(a, s, st);
    case 16: return dispatch_r<16, 0>(a, s, st);
    default: return dispatch_r<32, 0>(a, s, st);
    }
}
