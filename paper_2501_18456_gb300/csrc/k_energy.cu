// Energy scoring of large batches (Sec. 4.3, Eq. 1):
//     E(s) = -sum_i h_i(s_i) - sum_{i<j} J_ij(s_i, s_j),
// with the couplings streamed through shared memory once per pass of a CTA.
//
// A CTA owns up to 256*R sequences (their states in shared memory, rows
// padded to an odd number of 32-bit words).  For i = 0..L-2 a producer warp
// streams the slab Jg[i][i+1..L) (gather layout: block (i,j) holds J_ij(a,b)
// at b*q + a) in chunks of jc blocks through a ring of shared-memory stages
// with cp.async.bulk; every consumer thread owns R sequences and adds, for
// each staged block, the element at s_j*q + s_i of its sequences.  FP32 sums
// over j ascending within i ascending.  A sequence holding a symbol >= q is
// flagged and its energy is then unspecified (its symbols are read as 0).
// Every mbarrier wait is bounded by %globaltimer (2 s); a timeout sets bit 2
// of the model's device error word and leaves the energies unspecified.
#include "bm_internal.cuh"
#include "tc_common.cuh"

#include <algorithm>

namespace {

using namespace bmtc;

constexpr int kConsumerWarps = 8;
constexpr int kThreads = (kConsumerWarps + 1) * 32;
constexpr int kStages = 3;
constexpr size_t kStageTarget = 28 * 1024;
constexpr size_t kSmemBudget = 220 * 1024;

struct EnArgs {
    const float *h, *Jg;
    const uint8_t *S;
    float *E;
    int *bad, *err;
    int n, L, q, bs, jc, Ls, R;  // Ls: state row stride (bytes)
};

template <int R>
__global__ void __launch_bounds__(kThreads, 1) k_energy_staged(const EnArgs p)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const uint32_t stage_bytes = (uint32_t)p.jc * (uint32_t)p.bs * 4u;
    uint8_t *sv = smem + (size_t)kStages * stage_bytes;  // [256*R][Ls] states
    uint64_t *bars = reinterpret_cast<uint64_t *>(sv + (size_t)256 * R * p.Ls + 16 - ((size_t)256 * R * p.Ls) % 16);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(bars + 2 * kStages);
    const uint32_t full0 = su32(bars), empty0 = full0 + 8 * kStages;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int L = p.L, q = p.q;
    const long long per_cta = 256LL * R;
    const long long k0 = (long long)blockIdx.x * per_cta;
    const long long left = (long long)p.n - k0;
    const int nloc = (int)(left < per_cta ? left : per_cta);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, kConsumerWarps);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    int inval = 0;
    for (int t = threadIdx.x; t < nloc * L; t += blockDim.x) {
        const int c = t / L, x = t - c * L;
        uint8_t v = p.S[(size_t)(k0 + c) * L + x];
        if (v >= q) {
            inval = 1;
            v = 0;
        }
        sv[(size_t)c * p.Ls + x] = v;
    }
    if (__syncthreads_or(inval) && threadIdx.x == 0) atomicOr(p.bad, 1);

    if (warp == kConsumerWarps) {
        // ------------------------------------------------------- producer
        if (lane != 0) return;
        long long t = 0;
        bool ok = true;
        for (int i = 0; i + 1 < L && ok; ++i) {
            for (int j0 = i + 1; j0 < L; j0 += p.jc, ++t) {
                const int s = (int)(t % kStages);
                const long long use = t / kStages;
                if (use > 0 && !mbar_wait(empty0 + 8 * s, (uint32_t)((use - 1) & 1), abort_flag, p.err)) {
                    ok = false;
                    break;
                }
                const int nj = min(p.jc, L - j0);
                const uint32_t bytes = (uint32_t)nj * (uint32_t)p.bs * 4u;
                mbar_expect_tx(full0 + 8 * s, bytes);
                bulk_g2s(su32(smem + (size_t)s * stage_bytes), p.Jg + ((size_t)i * L + j0) * p.bs, bytes,
                         full0 + 8 * s);
            }
        }
        if (*abort_flag) {  // let the copies in flight land before exit
            volatile int no_abort = 0;
            for (long long u = t > kStages ? t - kStages : 0; u < t; ++u)
                mbar_wait(full0 + 8 * (int)(u % kStages), (uint32_t)((u / kStages) & 1), &no_abort, p.err);
        }
        return;
    }

    // ----------------------------------------------------------- consumers
    const int tid = warp * 32 + lane;  // 0..255
    float acc[R];
    const uint8_t *row[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int c = tid + 256 * r;
        row[r] = sv + (size_t)(c < nloc ? c : 0) * p.Ls;
        acc[r] = 0.0f;
        if (c < nloc)
            for (int i = 0; i < L; ++i) acc[r] -= p.h[i * q + row[r][i]];
    }
    const uint32_t stage0 = su32(smem);
    const uint32_t bstep = (uint32_t)p.bs * 4u, qb = (uint32_t)q * 4u;
    long long t = 0;
    bool ok = true;
    for (int i = 0; i + 1 < L && ok; ++i) {
        uint32_t si[R];
#pragma unroll
        for (int r = 0; r < R; ++r) si[r] = (uint32_t)row[r][i] * 4u;
        for (int j0 = i + 1; j0 < L; j0 += p.jc, ++t) {
            const int s = (int)(t % kStages);
            if (!mbar_wait(full0 + 8 * s, (uint32_t)((t / kStages) & 1), abort_flag, p.err)) {
                ok = false;
                break;
            }
            const int nj = min(p.jc, L - j0);
            const uint32_t base = stage0 + (uint32_t)s * stage_bytes;
            for (int jj = 0; jj < nj; ++jj) {
                const uint32_t blk = base + (uint32_t)jj * bstep;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    float v;
                    asm volatile("ld.shared.f32 %0, [%1];"
                                 : "=f"(v)
                                 : "r"(blk + (uint32_t)row[r][j0 + jj] * qb + si[r]));
                    acc[r] -= v;
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(empty0 + 8 * s);
        }
    }
    if (!ok) return;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int c = tid + 256 * r;
        if (c < nloc) p.E[k0 + c] = acc[r];
    }
}

}  // namespace

// Staged form for batches large enough to amortise one pass over J per CTA;
// returns BM_EINVAL when the shape does not fit (the caller then uses the
// gather form).
int bm_launch_energy_staged(const bm_model_s *m, const uint8_t *seqs, int n, float *E, int *bad, cudaStream_t st)
{
    const int L = m->L, q = m->q, bs = m->bs;
    const size_t row = (size_t)bs * 4;
    int jc = (int)(kStageTarget / row);
    jc = std::max(1, std::min(64, jc));
    const size_t stages = (size_t)kStages * jc * row;
    const int Ls = 4 * ((((L + 3) / 4)) | 1);  // odd number of words: conflict-free state rows
    int R = 4;
    while (R > 1 && stages + (size_t)256 * R * Ls + 16 + 2 * kStages * 8 + 16 > kSmemBudget) --R;
    const size_t smem = stages + (size_t)256 * R * Ls + 16 + 2 * kStages * 8 + 16;
    if (smem > kSmemBudget) return bm_fail(BM_EINVAL, "energy (staged): L=%d too large", L);
    EnArgs a;
    a.h = m->h;
    a.Jg = m->Jg;
    a.S = seqs;
    a.E = E;
    a.bad = bad;
    a.err = m->dflags + 3;
    a.n = n;
    a.L = L;
    a.q = q;
    a.bs = bs;
    a.jc = jc;
    a.Ls = Ls;
    a.R = R;
    const int grid = (int)(((long long)n + 256LL * R - 1) / (256LL * R));
    switch (R) {
    case 4:
        BM_CK(cudaFuncSetAttribute(k_energy_staged<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_energy_staged<4><<<grid, kThreads, smem, st>>>(a);
        break;
    case 3:
        BM_CK(cudaFuncSetAttribute(k_energy_staged<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_energy_staged<3><<<grid, kThreads, smem, st>>>(a);
        break;
    case 2:
        BM_CK(cudaFuncSetAttribute(k_energy_staged<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_energy_staged<2><<<grid, kThreads, smem, st>>>(a);
        break;
    default:
        BM_CK(cudaFuncSetAttribute(k_energy_staged<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_energy_staged<1><<<grid, kThreads, smem, st>>>(a);
    }
    BM_CK_LAUNCH("k_energy_staged");
    return BM_OK;
}
