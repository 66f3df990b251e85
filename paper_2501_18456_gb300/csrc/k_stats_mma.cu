// Chain pair counts on the 5th-generation tensor cores (tcgen05 + TMEM).
//
// The model statistics of Sec. 2.1 are the counts C[(i,a),(j,b)] =
// #{m : s_i^m = a, s_j^m = b} = (X^T X)[(i,a),(j,b)] with X the one-hot
// encoding of the chains, X[m][(i,a)] = [s_i^m == a].  That is a dense
// contraction over the chain index, so it runs as an MMA with exact 0/1
// operands and FP32 accumulation (exact for counts < 2^24).
//
// Tiling: an output tile is 128 rows (i,a) x 256 columns (j,b), i.e. TI =
// floor(128/q) row sites by TJ = floor(256/q) column sites; only tiles that
// hold some pair i <= j are computed.  The contraction dimension (chains)
// is cut into chunks of KT chains.  For each chunk all warps build the
// one-hot operand tiles in shared memory in the no-swizzle K-major
// canonical layout (core matrices of 8 rows x 16 bytes, K-adjacent cores 128
// bytes apart, 8-row groups 1024 bytes apart), one thread issues the MMAs
// (4 per chunk, K = 32 bytes each) into a 128 x 256 FP32 accumulator in
// TMEM, and commits them to the chunk's mbarrier, which releases the
// operand stage for the chunk after next.  The epilogue reads the
// accumulator with tcgen05.ld (warps 0-3, one TMEM lane = one row each),
// converts to int32 and writes the blocks with i <= j.
//
// Element type: E = 1 byte (FP8 E4M3, kind::f8f6f4, KT = 128 chains per
// chunk) or E = 2 bytes (BF16, kind::f16, KT = 64).  1.0 is exact in both.
#include "bm_internal.cuh"

#include <algorithm>

namespace {

constexpr int kRows = 128;         // MMA M
constexpr int kCols = 256;         // MMA N
constexpr int kRowBytes = 128;     // bytes of one operand row per chunk
constexpr int kThreads = 256;
constexpr int kStages = 2;
constexpr int kTileA = kRows * kRowBytes;  // 16 KB
constexpr int kTileB = kCols * kRowBytes;  // 32 KB
constexpr uint64_t kWaitNs = 2000000000ull;

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool mbar_try_parity(uint32_t bar, uint32_t parity)
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

// Bounded wait (2 s); on timeout records bit 1 in *err and returns false.
__device__ __forceinline__ bool mbar_wait_b(uint32_t bar, uint32_t parity, int *err)
{
    if (mbar_try_parity(bar, parity)) return true;
    const uint64_t t0 = gtimer();
    while (!mbar_try_parity(bar, parity))
        if (gtimer() - t0 > kWaitNs) {
            atomicOr(err, 2);
            return false;
        }
    return true;
}

// tcgen05 shared-memory matrix descriptor, no swizzle, K-major:
// start address >> 4 in bits 0-13, leading-dimension byte offset (distance
// of K-adjacent core matrices) >> 4 in bits 16-29, stride byte offset
// (distance of 8-row groups) >> 4 in bits 32-45, the fixed value 0b001 in
// bits 46-48, base offset 0, layout type 0 (no swizzle) in bits 61-63.
__device__ __forceinline__ uint64_t desc_noswizzle(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor: D format F32 (bits 4-5 = 1), A/B format in bits
// 7-9 / 10-12 (kind::f16: 1 = BF16; kind::f8f6f4: 0 = E4M3), both operands
// K-major (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
template <int E>
__host__ __device__ constexpr uint32_t idesc_counts()
{
    return (1u << 4) | ((E == 2 ? 1u : 0u) << 7) | ((E == 2 ? 1u : 0u) << 10) |
           ((uint32_t)(kCols >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);
}

template <int E>
__device__ __forceinline__ void mma_issue(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t id,
                                          uint32_t accum)
{
    if (E == 2) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
            "l"(ad), "l"(bd), "r"(id), "r"(accum));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
            "l"(ad), "l"(bd), "r"(id), "r"(accum));
    }
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// 4 chains' states -> per-byte 1 where the state equals a, else 0.
__device__ __forceinline__ uint32_t eq_bytes(uint32_t w, uint32_t a4)
{
    const uint32_t x = w ^ a4;
    const uint32_t t = ((x & 0x7f7f7f7fu) + 0x7f7f7f7fu) | x;
    return (~t & 0x80808080u) >> 7;
}

// One 16-byte operand chunk (8 BF16 or 16 FP8 values) for one row from the
// states of the chunk's chains at that row's site.
template <int E>
__device__ __forceinline__ uint4 onehot16(const uint32_t *sw, uint32_t a4)
{
    uint4 v;
    if (E == 1) {  // 16 chains, E4M3 1.0 = 0x38
        v.x = eq_bytes(sw[0], a4) * 0x38u;
        v.y = eq_bytes(sw[1], a4) * 0x38u;
        v.z = eq_bytes(sw[2], a4) * 0x38u;
        v.w = eq_bytes(sw[3], a4) * 0x38u;
    } else {  // 8 chains, BF16 1.0 = 0x3f80
        const uint32_t m0 = eq_bytes(sw[0], a4), m1 = eq_bytes(sw[1], a4);
        v.x = __byte_perm(m0, 0, 0x4140) * 0x3f80u;
        v.y = __byte_perm(m0, 0, 0x4342) * 0x3f80u;
        v.z = __byte_perm(m1, 0, 0x4140) * 0x3f80u;
        v.w = __byte_perm(m1, 0, 0x4342) * 0x3f80u;
    }
    return v;
}

// Byte offset of 16-byte chunk kc of row r in the no-swizzle K-major tile
// (8 chunks per row): core matrix (r/8, kc) at ((r/8)*8 + kc)*128, row r%8
// inside it at 16*(r%8).
__device__ __forceinline__ uint32_t tile_off(int r, int kc)
{
    return (uint32_t)((((r >> 3) << 3) + kc) << 7) + (uint32_t)((r & 7) << 4);
}

template <int E>
__global__ void __launch_bounds__(kThreads, 1) k_pair_counts_mma(const uint8_t *__restrict__ S, int M,
                                                                  int L, int q, int TI, int TJ,
                                                                  int32_t *__restrict__ counts, int *err)
{
    constexpr int KT = kRowBytes / E;  // chains per chunk
    const int rt = blockIdx.y, ct = blockIdx.x;
    const int i0 = rt * TI, j0 = ct * TJ;
    if (i0 >= L || j0 >= L || i0 > j0 + TJ - 1) return;  // no pair i <= j in this tile

    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *tileA = smem;                              // kStages x 16 KB
    unsigned char *tileB = smem + kStages * kTileA;           // kStages x 32 KB
    const int nsite = TI + TJ;                                // staged sites per chunk
    uint8_t *sT = smem + kStages * (kTileA + kTileB);         // kStages x [nsite][KT]
    uint64_t *bars = reinterpret_cast<uint64_t *>(sT + kStages * ((nsite * KT + 15) & ~15));
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + kStages + 1);  // [0] TMEM base, [1] ok flag
    const int tid = threadIdx.x, warp = tid >> 5;

    if (tid == 0) {
        for (int s = 0; s <= kStages; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(bars + s)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    const int nrow = TI * q, ncol = TJ * q;
    const int nchunks = (M + KT - 1) / KT;
    constexpr uint32_t idesc = idesc_counts<E>();
    volatile int *okflag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    if (tid == 0) *okflag = 1;
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
        const int s = c & 1;
        // Stage states (transposed: [site][chain]) for this chunk.
        uint8_t *st = sT + s * ((nsite * KT + 15) & ~15);
        const int m0 = c * KT;
        for (int k = tid; k < nsite * KT; k += kThreads) {
            const int x = k / KT, mm = k - x * KT;
            const int site = x < TI ? i0 + x : j0 + (x - TI);
            const int m = m0 + mm;
            st[k] = (m < M && site < L) ? S[(size_t)m * L + site] : 0xffu;  // 0xff never matches
        }
        // The MMAs of chunk c-2 read operand stage s; one thread waits for
        // their commit and the barrier below publishes the outcome.
        if (tid == 0 && c >= kStages && !mbar_wait_b(su32(bars + s), (uint32_t)(((c - kStages) >> 1) & 1), err))
            *okflag = 0;
        __syncthreads();
        if (!*okflag) {
            ok = false;
            break;
        }
        // One-hot operand tiles.
        unsigned char *A = tileA + s * kTileA, *B = tileB + s * kTileB;
        for (int k = tid; k < (kRows + kCols) * 8; k += kThreads) {
            const bool isA = k < kRows * 8;
            const int kk = isA ? k : k - kRows * 8;
            const int r = kk >> 3, kc = kk & 7;
            const int lim = isA ? nrow : ncol;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (r < lim) {
                const int x = (isA ? 0 : TI) + r / q;
                const uint32_t a4 = (uint32_t)(r % q) * 0x01010101u;
                const uint32_t *sw = reinterpret_cast<const uint32_t *>(st + x * KT + kc * (16 / E));
                v = onehot16<E>(sw, a4);
            }
            *reinterpret_cast<uint4 *>((isA ? A : B) + tile_off(r, kc)) = v;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = su32(A), b0 = su32(B);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {  // 4 MMAs x 32 bytes of K
                const uint64_t ad = desc_noswizzle(a0 + kk * 256, 128, 1024);
                const uint64_t bd = desc_noswizzle(b0 + kk * 256, 128, 1024);
                mma_issue<E>(tmem, ad, bd, idesc, (c > 0 || kk > 0) ? 1u : 0u);
            }
            mma_commit(su32(bars + s));
        }
    }
    // Wait for the last chunk's MMAs (the commit covers all earlier ones).
    if (tid == 0 && ok && nchunks > 0 &&
        !mbar_wait_b(su32(bars + ((nchunks - 1) & 1)), (uint32_t)(((nchunks - 1) >> 1) & 1), err))
        *okflag = 0;
    __syncthreads();
    ok = *okflag != 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok && warp < 4) {
        const int r = warp * 32 + (tid & 31);  // TMEM lane = row
        const int il = r / q, a = r % q;
        const int i = i0 + il;
        const bool row_ok = r < nrow && i < L;
        for (int col0 = 0; col0 < kCols; col0 += 32) {
            uint32_t v[32];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)col0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                  "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                  "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
                  "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
                  "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (!row_ok) continue;
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                const int cc = col0 + e;
                if (cc >= ncol) break;
                const int j = j0 + cc / q, b = cc % q;
                if (j >= L || j < i) continue;
                counts[bm_pair_block(L, i, j) * q * q + (size_t)a * q + b] = (int32_t)__uint_as_float(v[e]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
}

template <int E>
int launch_counts(const uint8_t *s, int M, int L, int q, int32_t *counts, int *err, cudaStream_t st)
{
    constexpr int KT = kRowBytes / E;
    const int TI = kRows / q, TJ = kCols / q;
    const int nsite = TI + TJ;
    const size_t smem = (size_t)kStages * (kTileA + kTileB) + (size_t)kStages * ((nsite * KT + 15) & ~15) +
                        (kStages + 1) * 8 + 16 + 1024;
    auto kern = k_pair_counts_mma<E>;
    BM_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((L + TJ - 1) / TJ, (L + TI - 1) / TI);
    kern<<<grid, kThreads, smem, st>>>(s, M, L, q, TI, TJ, counts, err);
    BM_CK_LAUNCH("k_pair_counts_mma");
    return BM_OK;
}

}  // namespace

int bm_launch_chain_stats_mma(const uint8_t *s, int M, int L, int q, int32_t *counts, int elem_bytes,
                              int *err, cudaStream_t st)
{
    if (M >= (1 << 24)) return bm_fail(BM_EINVAL, "chain_stats (tensor cores): M >= 2^24 not exact in FP32");
    return elem_bytes == 2 ? launch_counts<2>(s, M, L, q, counts, err, st)
                           : launch_counts<1>(s, M, L, q, counts, err, st);
}
