// Persistent-chain Gibbs sweeps with the local fields computed on the
// 5th-generation tensor cores (tcgen05 + TMEM + TMA).
//
// Method: Sec. 2.1 ("Monte Carlo estimation of the gradient"), sweep =
// every site once in order (Sec. 3.3).  The field of site i for chain m is
// H_i(a) = h_i(a) + sum_{j != i} J_ij(a, s_j), a contraction of the
// coupling rows (i,a) with the one-hot state X[m][(j,b)] = [s_j^m == b].
//
// Block-sequential exact Gibbs.  The sites are processed in blocks of B =
// floor(128/q) consecutive sites.  For a block, one MMA computes
//     G[(i,a), m] = sum_{(j,b)} J_ij(a,b) X0[m][(j,b)]
// for all its sites and all the CTA's chains from the states X0 at the start
// of the block (J_ii = 0, so site i's own state does not enter).  The sites
// of the block are then redrawn in order; for site i the sites j < i of the
// same block that already changed are corrected exactly,
//     H_i(a) = h_i(a) + G[(i,a), m] + sum_{j in block, j < i, s_j != s0_j}
//              (J_ij(a, s_j) - J_ij(a, s0_j)),
// which is the same conditional as sequential Gibbs (only the floating-point
// summation order differs).
//
// Precision.  J = J_hi + J_lo with J_hi = fp16(J) and J_lo = fp16(J - J_hi)
// (subnormals kept), two MMAs per K step accumulate into one FP32 TMEM
// accumulator; the one-hot operand is exact.  The representation error is
// <= 2^-22 |J| per coupling (plus 2^-25 absolute below fp16's normal
// range), i.e. FP32-class fields.
//
// Data path per CTA (one CTA per SM, NC chains, NC a multiple of 16):
//   warp 0     TMA producer: J_hi / J_lo tiles of 128 rows x 64 K (128-byte
//              rows, 128B swizzle) into a 3-stage ring, completion counted on
//              an mbarrier;
//   warp 1     allocates TMEM, one thread issues tcgen05.mma (M = 128 rows
//              (i,a), N = NC chains, K = 16 per instruction, hi and lo) and
//              commits each stage back to its producers;
//   warps 2-5  drawers: after the last chunk of a block read the accumulator
//              (tcgen05.ld, one TMEM lane = one row (i,a) per thread) into
//              shared memory, then redraw the block's sites, one thread per
//              chain, with the in-block corrections from coupling blocks
//              staged by bulk copies;
//   warps 6-9  generators: build the one-hot operand tile (NC rows x 64 K,
//              no swizzle) of each K chunk from the chain states in shared
//              memory, one thread per chain.
// Every mbarrier wait is bounded by %globaltimer (2 s); a timeout sets an
// abort flag and bit 2 of the model's device error word, every role leaves
// its loop, the producer waits (bounded) for its own copies, TMEM is
// released and the chains are left unchanged.
#include "bm_internal.cuh"

#include <cuda.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>

namespace {

constexpr int kNS = 3;                 // pipeline stages
constexpr int kKC = 64;                // fp16 K elements per chunk (128-byte rows)
constexpr int kRowsA = 128;            // MMA M
constexpr int kTileA = kRowsA * 128;   // bytes of one A tile (16 KB)
constexpr int kThreads = 320;          // 10 warps
constexpr int kBmax = 32;              // max sites per block
constexpr uint64_t kWaitNs = 2000000000ull;

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
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

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag, int *err)
{
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = gtimer();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (*abort_flag) return false;
        if (gtimer() - t0 > kWaitNs) {
            *abort_flag = 1;
            atomicOr(err, 4);
            return false;
        }
    }
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t n)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(n) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int x, int y, int z, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

// tcgen05 matrix descriptors (K-major).  Bits: start >> 4 [0,14), leading
// byte offset >> 4 [16,30), stride byte offset >> 4 [32,46), fixed 0b001 at
// [46,49), layout type [61,64) (0 = no swizzle, 2 = 128B swizzle).
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;            // leading offset (unused for 128B swizzle K-major)
    d |= (uint64_t)(1024 >> 4) << 32;  // 8-row groups 1024 bytes apart
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

__device__ __forceinline__ uint64_t desc_noswz(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(128 >> 4) << 16;   // K-adjacent core matrices 128 bytes apart
    d |= (uint64_t)(1024 >> 4) << 32;  // 8-row groups 1024 bytes apart
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}

__device__ __forceinline__ void named_bar(int id, int n)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// Byte offset of 16-byte piece p of row r in a no-swizzle K-major tile with
// 8 pieces per row: core matrix (r/8, p) at ((r/8)*8 + p)*128, row r%8 at +16*(r%8).
__device__ __forceinline__ uint32_t noswz_off(int r, int p)
{
    return (uint32_t)((((r >> 3) << 3) + p) << 7) + (uint32_t)((r & 7) << 4);
}

struct MmaArgs {
    const float *h;
    const float *Jg;  // gather layout (in-block corrections): Jg[i][j][b][a], block stride bs
    uint8_t *states;
    int *err;
    uint64_t seed, sweep0;
    float beta;
    int M, L, q, Lp, bs, B, nb, nK, NC, nsweeps;
    uint32_t tmem_cols, acc_stride;  // TMEM columns allocated; column offset of accumulator 1
};

// Row strides of the per-chain byte arrays, padded to an odd number of
// 32-bit words so that threads reading the same column of different chains
// hit different banks.
__host__ __device__ inline int st_stride(int Lp) { return Lp + 4; }
constexpr int kSnapStride = kBmax + 4;

// Shared-memory carve-up (offsets from the 1024-aligned base).
struct Smem {
    uint32_t a, b, hs, st, snap, corr, hrow, jtab, bars, misc, total;
};

__host__ __device__ inline Smem smem_layout(int NC, int Lp, int B, int bs, int nK)
{
    Smem s;
    s.a = 0;                                    // stage s: hi tile at +0, lo tile at +kTileA
    s.b = s.a + kNS * 2 * kTileA;
    s.hs = s.b + kNS * NC * 128;
    s.st = s.hs + kRowsA * (NC + 1) * 4;
    s.snap = s.st + NC * st_stride(Lp);         // 2 x [NC][kSnapStride]
    s.corr = (s.snap + 2 * NC * kSnapStride + 15) & ~15u;
    s.hrow = s.corr + (uint32_t)(B * (B - 1) / 2) * bs * 4;  // staged J_ij blocks, j < i in the block
    s.jtab = s.hrow + kRowsA * 4;                // block's h rows
    s.bars = (s.jtab + nK * 4 + 15) & ~15u;      // first/last site of each main chunk
    s.misc = s.bars + (3 * kNS + 7) * 8;
    s.total = s.misc + 16;
    return s;
}

// Block geometry shared by all roles: sites [i0, i0 + Bk) of block kb (global
// block counter over the launch), and the delta chunks that carry the
// previous block's changes: K chunks [d0, d0 + nD) covering its columns.
struct BlockGeo {
    int i0, Bk, pi0, pBk, d0, nD;
};

__device__ __forceinline__ BlockGeo block_geo(const MmaArgs &p, long long kb)
{
    BlockGeo g;
    const int blk = (int)(kb % p.nb);
    g.i0 = blk * p.B;
    g.Bk = min(p.B, p.L - g.i0);
    if (kb == 0) {
        g.pi0 = g.pBk = g.d0 = g.nD = 0;
    } else {
        const int pb = (int)((kb - 1) % p.nb);
        g.pi0 = pb * p.B;
        g.pBk = min(p.B, p.L - g.pi0);
        const int c_lo = g.pi0 * p.q, c_hi = (g.pi0 + g.pBk) * p.q;
        g.d0 = c_lo / kKC;
        g.nD = (c_hi - 1) / kKC - g.d0 + 1;
    }
    return g;
}

// Pipelined block-sequential sweep (see the file header).  Roles:
//   warp 0: TMA producer, warp 1: MMA issuer + TMEM owner,
//   warps 2-5: drawers (epilogue, redraws, snapshots),
//   warps 6-9: generators (one-hot and delta operand tiles).
// Per block kb the MMA consumes nK main chunks (X built from the states
// after block kb-2's redraw, with block kb-1 still at its old values) and
// nD delta chunks (+1 at the new, -1 at the old state of every site of block
// kb-1 that changed), so the accumulator holds the fields of block kb's
// sites for the states after block kb-1.  Accumulators alternate between
// two TMEM buffers; snap[kb % 2] holds block kb's states before its redraw.
__global__ void __launch_bounds__(kThreads, 1) k_gibbs_mma(const __grid_constant__ CUtensorMap tm_j,
                                                           const MmaArgs p)
{
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = su32(smem_raw);
    unsigned char *base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    const Smem lay = smem_layout(p.NC, p.Lp, p.B, p.bs, p.nK);
    float *Hs = reinterpret_cast<float *>(base + lay.hs);
    uint8_t *st = base + lay.st;
    uint8_t *snap = base + lay.snap;
    const float *corr = reinterpret_cast<const float *>(base + lay.corr);
    float *hrow = reinterpret_cast<float *>(base + lay.hrow);
    unsigned short *jtab = reinterpret_cast<unsigned short *>(base + lay.jtab);
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + lay.bars);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(base + lay.misc);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(base + lay.misc + 4);
    // barrier addresses
    const uint32_t full_a = su32(bars), full_b = full_a + 8 * kNS, empty = full_b + 8 * kNS;
    const uint32_t acc_full = empty + 8 * kNS;  // [2], one per accumulator buffer
    const uint32_t acc_empty = acc_full + 16;   // [2]
    const uint32_t ready = acc_empty + 16;      // [2], states after block kb: barrier kb % 2
    const uint32_t corr_bar = ready + 16;       // staged coupling blocks of block kb: phase kb
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = p.q, L = p.L, NC = p.NC, Lp = p.Lp;
    const int Sst = st_stride(Lp);
    const size_t cta0 = (size_t)blockIdx.x * NC;
    const long long nblocks = (long long)p.nsweeps * p.nb;

    if (tid == 0) {
        for (int s = 0; s < kNS; ++s) {
            mbar_init(full_a + 8 * s, 1);
            mbar_init(full_b + 8 * s, 4);
            mbar_init(empty + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(acc_full + 8 * b, 1);
            mbar_init(acc_empty + 8 * b, 4);
            mbar_init(ready + 8 * b, 4);
        }
        mbar_init(corr_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(p.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int k = tid; k < NC * Lp; k += kThreads) {
        const int c = k / Lp, x = k - c * Lp;
        const size_t m = cta0 + c;
        st[c * Sst + x] = (m < (size_t)p.M && x < L) ? p.states[m * L + x] : 0;
    }
    for (int c = tid; c < p.nK; c += kThreads) {  // sites touched by main chunk c
        const int k0 = c * kKC;
        jtab[2 * c] = (unsigned short)(k0 / q);
        jtab[2 * c + 1] = (unsigned short)min(L - 1, (k0 + kKC - 1) / q);
    }
    __syncthreads();
    {   // snapshot of block 0
        const int B0 = min(p.B, L);
        for (int k = tid; k < NC * B0; k += kThreads) {
            const int c = k / B0, x = k - c * B0;
            snap[c * kSnapStride + x] = st[c * Sst + x];
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    // Stage the coupling blocks J_ij (i, j in block kb, j < i) for the
    // in-block corrections: one bulk copy per block of bs floats.
    auto stage_corr = [&](long long kb) {
        const BlockGeo g = block_geo(p, kb);
        const uint32_t bytes = (uint32_t)(g.Bk * (g.Bk - 1) / 2) * (uint32_t)p.bs * 4u;
        mbar_expect_tx(corr_bar, bytes);
        int slot = 0;
        for (int pi = 1; pi < g.Bk; ++pi)
            for (int pj = 0; pj < pi; ++pj, ++slot)
                bulk_g2s(su32(base + lay.corr) + (uint32_t)slot * p.bs * 4u,
                         p.Jg + ((size_t)(g.i0 + pi) * L + (g.i0 + pj)) * p.bs, (uint32_t)p.bs * 4u, corr_bar);
    };

    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            long long t = 0;
            int s = 0, lap = 0;  // t = lap * kNS + s
            bool ok = true;
            for (long long kb = 0; kb < nblocks && ok; ++kb) {
                const BlockGeo g = block_geo(p, kb);
                for (int c = 0; c < p.nK + g.nD; ++c, ++t) {
                    if (lap > 0 && !mbar_wait(empty + 8 * s, (uint32_t)((lap - 1) & 1), abort_flag, p.err)) {
                        ok = false;
                        break;
                    }
                    const int x = (c < p.nK ? c : g.d0 + (c - p.nK)) * kKC;
                    mbar_expect_tx(full_a + 8 * s, 2 * kTileA);
                    // one op: slabs (hi, lo) of K chunk x/64 for 128 rows
                    tma_load_3d(su32(base + lay.a + s * 2 * kTileA), &tm_j, 0, g.i0 * q, 2 * (x / kKC), full_a + 8 * s);
                    if (++s == kNS) {
                        s = 0;
                        ++lap;
                    }
                }
            }
            if (*abort_flag) {
                volatile int no_abort = 0;
                for (long long u = t > kNS ? t - kNS : 0; u < t; ++u)
                    mbar_wait(full_a + 8 * (int)(u % kNS), (uint32_t)((u / kNS) & 1), &no_abort, p.err);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            // kind::f16: D F32 (bit 4), A = B = F16 (0), K-major, N >> 3 at 17, M >> 4 at 24.
            const uint32_t idesc = (1u << 4) | ((uint32_t)(NC >> 3) << 17) | ((uint32_t)(kRowsA >> 4) << 24);
            int s = 0;
            uint32_t ph = 0;  // stage and phase parity of the current chunk
            bool ok = true;
            for (long long kb = 0; kb < nblocks && ok; ++kb) {
                const BlockGeo g = block_geo(p, kb);
                const int buf = (int)(kb & 1);
                if (kb >= 2 && !mbar_wait(acc_empty + 8 * buf, (uint32_t)(((kb - 2) >> 1) & 1), abort_flag, p.err)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t dcol = tmem + (uint32_t)buf * p.acc_stride;
                for (int c = 0; c < p.nK + g.nD; ++c) {
                    if (!mbar_wait(full_a + 8 * s, ph, abort_flag, p.err) ||
                        !mbar_wait(full_b + 8 * s, ph, abort_flag, p.err)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t ah = su32(base + lay.a + s * 2 * kTileA), al = ah + kTileA;
                    const uint32_t bb = su32(base + lay.b + s * NC * 128);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint64_t bd = desc_noswz(bb + kk * 256);
                        mma_f16(dcol, desc_sw128(ah + kk * 32), bd, idesc, (c > 0 || kk > 0) ? 1u : 0u);
                        mma_f16(dcol, desc_sw128(al + kk * 32), bd, idesc, 1u);
                    }
                    mma_commit(empty + 8 * s);
                    if (++s == kNS) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
                if (!ok) break;
                mma_commit(acc_full + 8 * buf);
            }
        }
    } else if (warp < 6) {
        // ------------------------------------------------------------ drawers (warps 2-5)
        // Uniform control flow: every drawer runs the whole loop nest and meets
        // every named barrier; after an abort the work is skipped.
        const int w = tid - 64;            // 0..127
        const int lane_base = 32 * (warp & 3);
        const int row = lane_base + lane;  // TMEM lane / accumulator row read in the epilogue
        const unsigned HsStride = (unsigned)NC + 1;
        const uint32_t blkb = (uint32_t)p.bs;  // staged block stride (floats)
        bool ok = true;
        long long staged = 0;  // number of correction stagings issued (by w == 0)
        if (w == 0 && nblocks > 0) {
            stage_corr(0);
            staged = 1;
        }
        for (long long kb = 0; kb < nblocks; ++kb) {
            const BlockGeo g = block_geo(p, kb);
            const int buf = (int)(kb & 1);
            const uint64_t sweep = p.sweep0 + (uint64_t)(kb / p.nb);
            if (ok && !mbar_wait(acc_full + 8 * buf, (uint32_t)((kb >> 1) & 1), abort_flag, p.err)) ok = false;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int c0 = 0; c0 < NC && ok; c0 += 16) {
                uint32_t v[16];
                tmem_ld16(tmem + ((uint32_t)lane_base << 16) + (uint32_t)buf * p.acc_stride + (uint32_t)c0, v);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int e = 0; e < 16; ++e) Hs[row * HsStride + c0 + e] = __uint_as_float(v[e]);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(acc_empty + 8 * buf);
            for (int k = w; k < g.Bk * q; k += 128) hrow[k] = p.h[(size_t)g.i0 * q + k];
            if (ok && !mbar_wait(corr_bar, (uint32_t)(kb & 1), abort_flag, p.err)) ok = false;
            named_bar(1, 128);
            if (*abort_flag) ok = false;
            // --- sequential redraw of block kb, one thread per chain
            const uint8_t *old = snap + buf * NC * kSnapStride;
            for (int ch = w; ch < NC && ok; ch += 128) {
                const uint64_t m = cta0 + ch;
                for (int pp = 0; pp < g.Bk; ++pp) {
                    const int i = g.i0 + pp;
                    float H[32];
#pragma unroll
                    for (int a = 0; a < 32; ++a)
                        if (a < q) H[a] = hrow[pp * q + a] + Hs[(pp * q + a) * HsStride + ch];
                    const float *cb = corr + (uint32_t)(pp * (pp - 1) / 2) * blkb;  // blocks (i, j < i)
                    for (int jj = 0; jj < pp; ++jj) {
                        const int sn = st[ch * Sst + g.i0 + jj], so = old[ch * kSnapStride + jj];
                        if (sn == so) continue;
                        const float *rn = cb + jj * blkb + sn * q, *ro = cb + jj * blkb + so * q;
#pragma unroll
                        for (int a = 0; a < 32; ++a)
                            if (a < q) H[a] += rn[a] - ro[a];
                    }
                    float mx = -INFINITY;
#pragma unroll
                    for (int a = 0; a < 32; ++a)
                        if (a < q) {
                            H[a] *= p.beta;
                            mx = fmaxf(mx, H[a]);
                        }
                    float S = 0.0f;
#pragma unroll
                    for (int a = 0; a < 32; ++a)
                        if (a < q) {
                            S += expf(H[a] - mx);
                            H[a] = S;  // prefix sums
                        }
                    const uint32_t r24 = bm_u24(p.seed, m, sweep, (uint64_t)i, 0);
                    const float thr = ((float)r24 * 5.9604644775390625e-8f) * S;
                    int pick = q - 1;
#pragma unroll
                    for (int a = 31; a >= 0; --a)
                        if (a < q && thr < H[a]) pick = a;
                    st[ch * Sst + i] = (uint8_t)pick;
                }
            }
            // snapshot of the next block's states before its redraw
            if (ok && kb + 1 < nblocks) {
                const BlockGeo gn = block_geo(p, kb + 1);
                uint8_t *nsnap = snap + (buf ^ 1) * NC * kSnapStride;
                for (int k = w; k < NC * gn.Bk; k += 128) {
                    const int ch = k / gn.Bk, x = k - ch * gn.Bk;
                    nsnap[ch * kSnapStride + x] = st[ch * Sst + gn.i0 + x];
                }
            }
            named_bar(1, 128);
            // the staged blocks are free again: stage the next block's
            if (w == 0 && ok && !*abort_flag && kb + 1 < nblocks) {
                stage_corr(kb + 1);
                ++staged;
            }
            if (lane == 0) mbar_arrive(ready + 8 * buf);
        }
        if (!ok) *abort_flag = 1;
        if (w == 0 && *abort_flag && staged > 0) {
            volatile int no_abort = 0;  // let the last staging copies land before exit
            mbar_wait(corr_bar, (uint32_t)((staged - 1) & 1), &no_abort, p.err);
        }
    } else {
        // ------------------------------------------------------------ generators (warps 6-9)
        // Thread w owns the operand row of chain w (NC <= 128): per K chunk it
        // zeroes the row (8 x 16-byte stores) and then stores the few nonzero
        // halfwords (same thread, so program order keeps the stores ordered).
        // A main chunk holds +1 at (j, s_j) for the sites j it overlaps; a
        // delta chunk holds +1 at (j, new s_j) and -1 at (j, old s_j) for the
        // changed sites of the previous block.
        const int w = tid - 192;  // 0..127
        const bool own = w < NC;
        unsigned char *const row0 = base + lay.b + noswz_off(own ? w : 0, 0);
        const uint8_t *const strow = st + (own ? w : 0) * Sst;
        int s = 0, lap = 0;  // stage and ring lap of the current chunk
        bool ok = true;
        for (long long kb = 0; kb < nblocks && ok; ++kb) {
            const BlockGeo g = block_geo(p, kb);
            const int buf = (int)(kb & 1);
            // main chunks need the states after block kb-2; block kb-1 from its snapshot
            if (kb >= 2 && !mbar_wait(ready + 8 * buf, (uint32_t)(((kb - 2) >> 1) & 1), abort_flag, p.err)) {
                ok = false;
                break;
            }
            const uint8_t *psrow = snap + (buf ^ 1) * NC * kSnapStride + (own ? w : 0) * kSnapStride;
            const int pi0 = kb > 0 ? g.pi0 : L, pi1 = kb > 0 ? g.pi0 + g.pBk : L;  // block kb-1's sites
            for (int c = 0; c < p.nK + g.nD; ++c) {
                const bool delta = c >= p.nK;
                if (c == p.nK &&
                    !mbar_wait(ready + 8 * (buf ^ 1), (uint32_t)(((kb - 1) >> 1) & 1), abort_flag, p.err)) {
                    ok = false;
                    break;
                }
                if (lap > 0 && !mbar_wait(empty + 8 * s, (uint32_t)((lap - 1) & 1), abort_flag, p.err)) {
                    ok = false;
                    break;
                }
                const int k0 = (delta ? g.d0 + (c - p.nK) : c) * kKC;
                unsigned char *rowp = row0 + s * NC * 128;
                if (own) {
#pragma unroll
                    for (int pc = 0; pc < 8; ++pc)
                        *reinterpret_cast<uint4 *>(rowp + pc * 128) = make_uint4(0, 0, 0, 0);
                    if (!delta) {
                        const int jlo = jtab[2 * c], jhi = jtab[2 * c + 1];
                        for (int j = jlo; j <= jhi; ++j) {
                            const int sj = (j >= pi0 && j < pi1) ? psrow[j - pi0] : strow[j];
                            const int pos = j * q + sj - k0;
                            if (pos >= 0 && pos < kKC)
                                *reinterpret_cast<unsigned short *>(rowp + (pos >> 3) * 128 + (pos & 7) * 2) = 0x3c00u;
                        }
                    } else {
                        for (int x = 0; x < g.pBk; ++x) {
                            const int j = g.pi0 + x;
                            const int sn = strow[j], so = psrow[x];
                            if (sn == so) continue;
                            const int pn = j * q + sn - k0, po = j * q + so - k0;
                            if (pn >= 0 && pn < kKC)
                                *reinterpret_cast<unsigned short *>(rowp + (pn >> 3) * 128 + (pn & 7) * 2) = 0x3c00u;
                            if (po >= 0 && po < kKC)
                                *reinterpret_cast<unsigned short *>(rowp + (po >> 3) * 128 + (po & 7) * 2) = 0xbc00u;
                        }
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(full_b + 8 * s);
                if (++s == kNS) {
                    s = 0;
                    ++lap;
                }
            }
        }
        if (!ok) *abort_flag = 1;
    }
    // Roles that stopped early (abort) still arrive here; nothing of the
    // pipeline is waited on past this point.
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.tmem_cols)
                     : "memory");
    if (*abort_flag) return;
    for (int k = tid; k < NC * L; k += kThreads) {
        const int c = k / L, x = k - c * L;
        const size_t m = cta0 + c;
        if (m < (size_t)p.M) p.states[m * L + x] = st[c * Sst + x];
    }
}

// Jt[L*q rows (i,a)][Kp/64 slabs][2 (hi, lo)][64] fp16: for column
// k = (j,b) of slab k/64, hi = fp16(J_ij(a,b)) and lo = fp16(J_ij(a,b) - hi)
// (J_ij(a,b) = J[i][j][a][b]); zero padding beyond L*q columns.  Each row
// interleaves the hi and lo slabs so one 3-D TMA op brings both.
__global__ void k_build_mma_layout(const float *__restrict__ J, __half *__restrict__ jt, int L, int q, int Kp)
{
    const size_t rows = (size_t)L * q, n = rows * Kp;
    const int Q = L * q;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        const size_t r = t / Kp;
        const int k = (int)(t - r * Kp);
        float v = 0.0f;
        if (k < Q) {
            const int i = (int)(r / q), a = (int)(r % q), j = k / q, b = k % q;
            v = J[(((size_t)i * L + j) * q + a) * q + b];
        }
        const __half vh = __float2half_rn(v);
        const size_t o = r * (size_t)(2 * Kp) + (size_t)(k / kKC) * (2 * kKC) + (k % kKC);
        jt[o] = vh;
        jt[o + kKC] = __float2half_rn(v - __half2float(vh));
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(f);
    });
    return fn;
}

// 3-D view of Jt: dim 0 = 64 elements of a slab (contiguous), dim 1 = row
// (stride 2*Kp*2 bytes), dim 2 = slab index 2*(k/64) + {0 hi, 1 lo} (stride
// 128 bytes).  Box {64, 128, 2}: one op lands the hi tile and then the lo
// tile of a K chunk for 128 rows, each a 128B-swizzled 128 x 64 tile.
int make_map(CUtensorMap *map, const __half *ptr, int rows, int Kp)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return bm_fail(BM_ECUDA, "cuTensorMapEncodeTiled entry point unavailable");
    cuuint64_t dims[3] = {(cuuint64_t)kKC, (cuuint64_t)rows, (cuuint64_t)(2 * Kp / kKC)};
    cuuint64_t strides[2] = {(cuuint64_t)Kp * 4, (cuuint64_t)kKC * 2};
    cuuint32_t box[3] = {(cuuint32_t)kKC, (cuuint32_t)kRowsA, 2};
    cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, const_cast<__half *>(ptr), dims, strides, box,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return bm_fail(BM_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return BM_OK;
}

}  // namespace

// Chains per CTA for the tensor-core sweep (multiple of 16, <= 128), or 0
// when the shape does not fit one CTA's shared memory.
int bm_gibbs_mma_chains_per_cta(const bm_model_s *m, int M)
{
    if (m->L > 65535) return 0;  // site indices of the chunk table are 16-bit
    const int nsm = m->num_sms > 0 ? m->num_sms : 1;
    int nc = (M + nsm - 1) / nsm;
    nc = std::max(16, (nc + 15) & ~15);
    nc = std::min(nc, 128);  // one operand-row generator thread per chain
    const int Lp = (m->L + 15) & ~15;
    const int B = std::min(kBmax, kRowsA / m->q);
    const int nK = (m->L * m->q + kKC - 1) / kKC;
    while (nc >= 16 && smem_layout(nc, Lp, B, m->bs, nK).total + 1024 > 227 * 1024) nc -= 16;
    return nc >= 16 ? nc : 0;
}

int bm_mma_prepare(bm_model_s *m, cudaStream_t st)
{
    const int rows = m->L * m->q;
    const int Kp = (rows + kKC - 1) / kKC * kKC;
    if (!m->Jt) {
        m->Kp = Kp;
        BM_CK(cudaMalloc(&m->Jt, (size_t)rows * Kp * 2 * sizeof(__half)));
        const int rc = make_map(reinterpret_cast<CUtensorMap *>(m->tmap_j), (const __half *)m->Jt, rows, Kp);
        if (rc != BM_OK) return rc;
    }
    const size_t n = (size_t)rows * Kp;
    const int grid = (int)std::min<size_t>((n + 255) / 256, 152 * 64);
    k_build_mma_layout<<<grid, 256, 0, st>>>(m->J, (__half *)m->Jt, m->L, m->q, Kp);
    BM_CK_LAUNCH("k_build_mma_layout");
    m->mma_current = true;
    return BM_OK;
}

int bm_launch_gibbs_mma(bm_model_s *m, bm_chains_s *c, int nsweeps, float beta, cudaStream_t st)
{
    const int NC = bm_gibbs_mma_chains_per_cta(m, c->M);
    if (NC == 0) return bm_fail(BM_EINVAL, "tensor-core sweep: shape does not fit shared memory");
    if (!m->mma_current) {
        const int rc = bm_mma_prepare(m, st);
        if (rc != BM_OK) return rc;
    }
    MmaArgs a;
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
    a.B = std::min(kBmax, kRowsA / c->q);
    a.nb = (c->L + a.B - 1) / a.B;
    a.nK = m->Kp / kKC;
    a.NC = NC;
    a.nsweeps = nsweeps;
    a.acc_stride = NC <= 32 ? 32 : NC <= 64 ? 64 : NC <= 128 ? 128 : 256;
    a.tmem_cols = 2 * a.acc_stride;  // two accumulators
    const Smem lay = smem_layout(NC, a.Lp, a.B, a.bs, a.nK);
    const size_t smem = lay.total + 1024;
    BM_CK(cudaFuncSetAttribute(k_gibbs_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = (c->M + NC - 1) / NC;
    k_gibbs_mma<<<grid, kThreads, smem, st>>>(*reinterpret_cast<const CUtensorMap *>(m->tmap_j), a);
    BM_CK_LAUNCH("k_gibbs_mma");
    return BM_OK;
}
