// Persistent-chain Gibbs sweeps with the local fields computed on the
// 5th-generation tensor cores (tcgen05 + TMEM + TMA).
//
// Method: Sec. 2.1 ("Monte Carlo estimation of the gradient"), sweep =
// every site once in order (Sec. 3.3).  The field of site i for chain m is
// H_i(a) = h_i(a) + sum_{j != i} J_ij(a, s_j), a contraction of the
// coupling rows (i,a) with the one-hot state X[m][(j,b)] = [s_j^m == b].
//
// Block-sequential exact Gibbs.  The sites are processed in blocks of B <=
// floor(128/q) consecutive sites (block_sites: the block's in-block coupling
// blocks must also fit 32 KB of staging; global block counter kb over the launch,
// block kb covers sites of block kb mod nb of sweep kb / nb).  The MMAs
// compute, for the 128 rows (i,a) of a block and all the CTA's chains,
//     G[(i,a), m] = sum_{(j,b)} J_ij(a,b) X[m][(j,b)]
// for the states at the start of the block (J_ii = 0, so site i's own state
// does not enter).  The block's sites are then redrawn in order; for site i
// the sites j < i of the same block that already changed are corrected
// exactly, H_i(a) = h_i(a) + G[(i,a), m] + sum (J_ij(a, s_j) - J_ij(a, s0_j)),
// which is the same conditional as sequential Gibbs (only the floating-point
// summation order differs).
//
// Paired blocks.  Blocks are taken in pairs P = (2P, 2P+1).  One one-hot
// operand tile of a K chunk feeds the MMAs of both blocks of the pair, which
// halves the operand generation per flop.  Schedule of pair P (each step a
// run of 64-column K chunks):
//   A  main chunks [0, X) into both accumulators, built from the states
//      after block 2P-3 with blocks 2P-2 and 2P-1 taken from their
//      pre-redraw snapshots (those two blocks are being redrawn meanwhile);
//   B  delta chunks of block 2P-2 (+1 at the new, -1 at the old state of
//      each changed site) into block 2P-1's accumulator, which completes it;
//   C  main chunks [X, nK) into both accumulators;
//   D  delta chunks of blocks 2P-2 and 2P-1 into both accumulators, which
//      completes block 2P (block 2P+1 is completed by step B of pair P+1).
// So block 2P sees the states after 2P-1 and block 2P+1 those after 2P.
//
// Precision.  J = J_hi + J_lo with J_hi = fp16(J) and J_lo = fp16(J - J_hi)
// (subnormals kept), two MMAs per K step accumulate into one FP32 TMEM
// accumulator; the one-hot operand is exact.  The representation error is
// <= 2^-22 |J| per coupling (plus 2^-25 absolute below fp16's normal
// range), i.e. FP32-class fields.
//
// Data path per CTA (one CTA per SM, NC <= 128 chains, NC a multiple of 16):
//   warp 0     TMA producer: J_hi / J_lo tiles of 128 rows x 64 K (128-byte
//              rows, 128B swizzle) of both blocks of the pair into a 2-slot
//              ring, one 64 KB copy when the two blocks are consecutive
//              (the layout pads every block to 128 rows);
//   warp 1     allocates TMEM (four accumulators, block kb in slot kb % 4),
//              one thread issues tcgen05.mma (M = 128 rows (i,a), N = NC
//              chains, K = 16 per instruction, hi and lo) and commits each
//              ring slot back to its producer;
//   warps 2-5  drawers: per site, read its q accumulator rows (tcgen05.ld,
//              one TMEM lane = one row (i,a) per thread), add h and store
//              them as one padded row per chain; then redraw the site, one
//              thread per chain, reading its row and the in-block coupling
//              blocks (padded layout Jc, one bulk copy per block) with
//              128-bit loads; they also take the snapshots;
//   warps 6-9  generators: build the one-hot operand tile (NC rows x 64 K,
//              no swizzle) of each K chunk into a 3-slot ring, one thread
//              per chain.
// Every mbarrier wait is bounded by %globaltimer (2 s); a timeout sets an
// abort flag and bit 2 of the model's device error word, every role leaves
// its loop, the producer waits (bounded) for its own copies, TMEM is
// released and the chains are left unchanged.
#include "bm_internal.cuh"

#include <type_traits>
#include "tc_common.cuh"

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>

using namespace bmtc;

namespace {

constexpr int kNA = 2;                 // coupling-tile ring slots (hi and lo of two blocks, 64 KB each)
constexpr int kNB = 3;                 // one-hot tile ring slots (NC x 128 bytes each)
constexpr int kKC = 64;                // fp16 K elements per chunk (128-byte rows)
constexpr int kRowsA = 128;            // MMA M
constexpr int kTileA = kRowsA * 128;   // bytes of one hi or lo tile (16 KB)
constexpr int kSlotA = 4 * kTileA;     // ring slot: [hi, lo][block 0, block 1] tiles
constexpr int kThreads = 320;          // 10 warps
constexpr int kBmax = 32;              // max sites per block
constexpr int kNBars = 2 * kNA + 2 * kNB + 4 + 4 + 2 + 1;
struct MmaArgs {
    const float *h;
    const float *Jc;  // in-block coupling blocks: [site block][pair slot][b][a padded to q4]
    uint8_t *states;
    int *err;
    uint64_t seed, sweep0, chain0;  // chain0: global index of chain 0 (Philox counter)
    float beta_l2e;  // beta * log2(e): weights exp(beta H) = 2^(beta log2(e) H)
    int M, L, q, Lp, bs, B, nb, nK, X, NC, nsweeps;
    long long nblocks;
    uint32_t tmem_cols, acc_stride;  // TMEM columns allocated; columns per accumulator
};

// Row strides of the per-chain byte arrays, padded to an odd number of
// 32-bit words so that threads reading the same column of different chains
// hit different banks.
__host__ __device__ inline int st_stride(int Lp) { return Lp + 4; }
__host__ __device__ inline int snap_stride(int B) { return 4 * (((B + 3) / 4) | 1); }
__host__ __device__ inline int q4_of(int q) { return (q + 3) & ~3; }
// Row stride (floats) of the staged fields, one row per chain: q rounded up
// to 4, plus 4 when that is an even number of 16-byte units, so that eight
// consecutive rows start in eight different 16-byte bank groups.
__host__ __device__ inline int hs_stride(int q) { return ((q4_of(q) >> 2) & 1) ? q4_of(q) : q4_of(q) + 4; }

// Shared-memory carve-up (offsets from the 1024-aligned base).
struct Smem {
    uint32_t a, b, hs, st, snap, corr, hrow, jtab, bars, misc, total;
};

__host__ __device__ inline Smem smem_layout(int NC, int Lp, int B, int q, int nK)
{
    Smem s;
    s.a = 0;                                      // slot: hi tiles at +0, +kTileA; lo at +2, +3 kTileA
    s.b = s.a + kNA * kSlotA;
    s.hs = s.b + kNB * NC * 128;
    s.st = s.hs + NC * hs_stride(q) * 4;          // fields h + G of one site: [chain][a]
    s.snap = s.st + NC * st_stride(Lp);           // [2 pair slots][2 blocks][NC][snap_stride]
    s.corr = (s.snap + 4 * NC * snap_stride(B) + 15) & ~15u;
    s.hrow = s.corr + (uint32_t)(B * (B - 1) / 2) * q * q4_of(q) * 4;  // staged J_ij blocks, j < i in the block
    s.jtab = s.hrow + kRowsA * 4;                 // block's h rows
    s.bars = (s.jtab + nK * 4 + 15) & ~15u;       // first/last site of each K chunk
    s.misc = s.bars + kNBars * 8;
    s.total = s.misc + 16;
    return s;
}

// Sites [i0, i0 + Bk) of block kb.
struct Blk {
    int i0, Bk;
};

__device__ __forceinline__ Blk blk_of(const MmaArgs &p, long long kb)
{
    Blk g;
    g.i0 = (int)(kb % p.nb) * p.B;
    g.Bk = min(p.B, p.L - g.i0);
    return g;
}

// One step of a pair's schedule: n K chunks (n0 from c0, then the rest from
// c1), their kind (main or delta), the blocks whose accumulators they feed
// (t1 < 0: one), the block whose redraw the generator waits for before the
// step, the block whose accumulator is complete after it, and the blocks
// whose changes a delta step carries (d1 < 0: one).
struct Seg {
    int n, n0, c0, c1;
    bool delta;
    long long t0, t1, wait_kb, commit_kb, d0, d1;
};

__device__ __forceinline__ int seg_chunk(const Seg &s, int k) { return k < s.n0 ? s.c0 + k : s.c1 + (k - s.n0); }

__device__ __forceinline__ void blk_chunks(const MmaArgs &p, long long kb, int &lo, int &hi)
{
    const Blk g = blk_of(p, kb);
    lo = g.i0 * p.q / kKC;
    hi = ((g.i0 + g.Bk) * p.q - 1) / kKC;
}

__device__ Seg seg_info(const MmaArgs &p, long long P, int step)
{
    Seg s;
    s.n = s.n0 = s.c0 = s.c1 = 0;
    s.delta = false;
    s.t0 = s.t1 = s.wait_kb = s.commit_kb = s.d0 = s.d1 = -1;
    const long long b0 = 2 * P, b1 = 2 * P + 1;
    const bool has0 = b0 < p.nblocks, has1 = b1 < p.nblocks;
    if (step == 0 || step == 2) {  // main chunks
        if (!has0) return s;
        s.c0 = step == 0 ? 0 : p.X;
        s.n = s.n0 = step == 0 ? p.X : p.nK - p.X;
        s.t0 = b0;
        s.t1 = has1 ? b1 : -1;
        if (step == 2 && P == 0) s.commit_kb = b0;
        return s;
    }
    if (P < 1) return s;
    s.delta = true;
    if (step == 1) {  // block 2P-2's changes into block 2P-1
        if (b0 - 1 >= p.nblocks) return s;
        int lo, hi;
        blk_chunks(p, b0 - 2, lo, hi);
        s.c0 = lo;
        s.n = s.n0 = hi - lo + 1;
        s.t0 = b0 - 1;
        s.d0 = b0 - 2;
        s.wait_kb = b0 - 2;
        s.commit_kb = b0 - 1;
        return s;
    }
    if (!has0) return s;  // step 3: blocks 2P-2, 2P-1 into the pair
    int a0, a1, c0, c1;
    blk_chunks(p, b0 - 2, a0, a1);
    blk_chunks(p, b0 - 1, c0, c1);
    if (c0 <= a1 + 1 && a0 <= c1 + 1) {  // overlapping or adjacent ranges: one run
        s.c0 = min(a0, c0);
        s.n = s.n0 = max(a1, c1) - s.c0 + 1;
    } else {  // the pair of blocks wraps around the end of a sweep
        s.c0 = a0;
        s.n0 = a1 - a0 + 1;
        s.c1 = c0;
        s.n = s.n0 + (c1 - c0 + 1);
    }
    s.t0 = b0;
    s.t1 = has1 ? b1 : -1;
    s.d0 = b0 - 2;
    s.d1 = b0 - 1;
    s.wait_kb = b0 - 1;
    s.commit_kb = b0;
    return s;
}

// Persistent paired-block sweep (see the file header).
__global__ void __launch_bounds__(kThreads, 1) k_gibbs_mma(const __grid_constant__ CUtensorMap tm_j2,
                                                           const __grid_constant__ CUtensorMap tm_j1,
                                                           const MmaArgs p)
{
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = su32(smem_raw);
    unsigned char *base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    const Smem lay = smem_layout(p.NC, p.Lp, p.B, p.q, p.nK);
    float *Hs = reinterpret_cast<float *>(base + lay.hs);
    uint8_t *st = base + lay.st;
    uint8_t *snap = base + lay.snap;
    const float4 *corr4 = reinterpret_cast<const float4 *>(base + lay.corr);
    float *hrow = reinterpret_cast<float *>(base + lay.hrow);
    unsigned short *jtab = reinterpret_cast<unsigned short *>(base + lay.jtab);
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + lay.bars);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(base + lay.misc);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(base + lay.misc + 4);
    // barrier addresses
    const uint32_t full_a = su32(bars), empty_a = full_a + 8 * kNA;
    const uint32_t full_b = empty_a + 8 * kNA, empty_b = full_b + 8 * kNB;
    const uint32_t acc_full = empty_b + 8 * kNB;  // [4], accumulator of block kb in slot kb % 4
    const uint32_t acc_empty = acc_full + 32;     // [4]
    const uint32_t ready = acc_empty + 32;        // [2], states after block kb: barrier kb % 2
    const uint32_t corr_bar = ready + 16;         // staged coupling blocks of block kb: phase kb
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = p.q, L = p.L, NC = p.NC, Lp = p.Lp;
    const int Sst = st_stride(Lp), Ssn = snap_stride(p.B);
    const size_t cta0 = (size_t)blockIdx.x * NC;
    const long long nblocks = p.nblocks;
    const long long npairs = (nblocks + 1) / 2;  // the schedule runs P = 0 .. npairs (tail)
    // snapshot of block kb (its states before its redraw): pair slot (kb/2)%2, block kb%2
    auto snap_of = [&](long long kb) { return snap + (size_t)((((kb >> 1) & 1) * 2 + (kb & 1)) * NC) * Ssn; };

    if (tid == 0) {
        for (int s = 0; s < kNA; ++s) {
            mbar_init(full_a + 8 * s, 1);
            mbar_init(empty_a + 8 * s, 1);
        }
        for (int s = 0; s < kNB; ++s) {
            mbar_init(full_b + 8 * s, 4);
            mbar_init(empty_b + 8 * s, 1);
        }
        for (int b = 0; b < 4; ++b) {
            mbar_init(acc_full + 8 * b, 1);
            mbar_init(acc_empty + 8 * b, 4);
        }
        mbar_init(ready, 4);
        mbar_init(ready + 8, 4);
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
    for (int c = tid; c < p.nK; c += kThreads) {  // sites touched by K chunk c
        const int k0 = c * kKC;
        jtab[2 * c] = (unsigned short)min(L - 1, k0 / q);
        jtab[2 * c + 1] = (unsigned short)min(L - 1, (k0 + kKC - 1) / q);
    }
    __syncthreads();
    for (long long kb = 0; kb < 2 && kb < nblocks; ++kb) {  // snapshots of pair 0
        const Blk g = blk_of(p, kb);
        uint8_t *sn = snap_of(kb);
        for (int k = tid; k < NC * g.Bk; k += kThreads) {
            const int c = k / g.Bk, x = k - c * g.Bk;
            sn[c * Ssn + x] = st[c * Sst + g.i0 + x];
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    // Stage the coupling blocks J_ij (i, j in block kb, j < i) for the
    // in-block corrections: one bulk copy per block of bs floats.
    // Stage the in-block coupling blocks of block kb (its pairs pi > pj are
    // the first Bk(Bk-1)/2 slots of its Jc entry): one bulk copy.
    auto stage_corr = [&](long long kb) {
        const Blk g = blk_of(p, kb);
        const uint32_t row = (uint32_t)q * (uint32_t)q4_of(q);
        const uint32_t bytes = (uint32_t)(g.Bk * (g.Bk - 1) / 2) * row * 4u;
        mbar_expect_tx(corr_bar, bytes);
        if (bytes > 0)
            bulk_g2s(su32(base + lay.corr), p.Jc + (size_t)(kb % p.nb) * (p.B * (p.B - 1) / 2) * row, bytes,
                     corr_bar);
    };

    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            long long issued = 0;
            int sa = 0, lap = 0;  // ring slot and lap of the next coupling tile
            bool ok = true;
            for (long long P = 0; P <= npairs && ok; ++P)
                for (int step = 0; step < 4 && ok; ++step) {
                    const Seg sg = seg_info(p, P, step);
                    for (int k = 0; k < sg.n && ok; ++k) {
                        const int c = seg_chunk(sg, k);
                        if (lap > 0 && !mbar_wait(empty_a + 8 * sa, (uint32_t)((lap - 1) & 1), abort_flag, p.err)) {
                            ok = false;
                            break;
                        }
                        const int nt = sg.t1 >= 0 ? 2 : 1;
                        const int r0 = (int)(sg.t0 % p.nb) * kRowsA, r1 = (int)((sg.t1 >= 0 ? sg.t1 : 0) % p.nb) * kRowsA;
                        const uint32_t dst = su32(base + lay.a + sa * kSlotA), bar = full_a + 8 * sa;
                        mbar_expect_tx(bar, (uint32_t)nt * 2 * kTileA);
                        if (nt == 2 && r1 == r0 + kRowsA) {
                            // one op: hi and lo slabs of K chunk c for both blocks' 256 rows
                            tma_load_3d(dst, &tm_j2, 0, r0, 2 * c, bar);
                        } else {
                            for (int u = 0; u < nt; ++u) {
                                const int r = u == 0 ? r0 : r1;
                                tma_load_3d(dst + u * kTileA, &tm_j1, 0, r, 2 * c, bar);                // hi
                                tma_load_3d(dst + (2 + u) * kTileA, &tm_j1, 0, r, 2 * c + 1, bar);      // lo
                            }
                        }
                        ++issued;
                        if (++sa == kNA) {
                            sa = 0;
                            ++lap;
                        }
                    }
                }
            if (*abort_flag) {
                volatile int no_abort = 0;
                for (long long u = issued > kNA ? issued - kNA : 0; u < issued; ++u)
                    mbar_wait(full_a + 8 * (int)(u % kNA), (uint32_t)((u / kNA) & 1), &no_abort, p.err);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            // kind::f16: D F32 (bit 4), A = B = F16 (0), K-major, N >> 3 at 17, M >> 4 at 24.
            const uint32_t idesc = (1u << 4) | ((uint32_t)(NC >> 3) << 17) | ((uint32_t)(kRowsA >> 4) << 24);
            int sa = 0, sb = 0;
            uint32_t pha = 0, phb = 0;
            bool ok = true;
            for (long long P = 0; P <= npairs && ok; ++P)
                for (int step = 0; step < 4 && ok; ++step) {
                    const Seg sg = seg_info(p, P, step);
                    for (int k = 0; k < sg.n && ok; ++k) {
                        const int c = seg_chunk(sg, k);
                        const bool first = !sg.delta && c == 0;  // first chunk of the pair's accumulators
                        if (!mbar_wait(full_b + 8 * sb, phb, abort_flag, p.err)) {
                            ok = false;
                            break;
                        }
                        if (!mbar_wait(full_a + 8 * sa, pha, abort_flag, p.err)) {
                            ok = false;
                            break;
                        }
                        const uint32_t bb = su32(base + lay.b + sb * NC * 128);
                        const uint32_t slot_a = su32(base + lay.a + sa * kSlotA);
                        for (int u = 0; u < 2; ++u) {
                            const long long tb = u == 0 ? sg.t0 : sg.t1;
                            if (tb < 0) continue;
                            if (first && tb >= 4 &&
                                !mbar_wait(acc_empty + 8 * (int)(tb & 3), (uint32_t)(((tb - 4) >> 2) & 1), abort_flag,
                                           p.err)) {
                                ok = false;
                                break;
                            }
                            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                            const uint32_t dcol = tmem + (uint32_t)(tb & 3) * p.acc_stride;
                            const uint32_t ah = slot_a + u * kTileA, al = slot_a + (2 + u) * kTileA;
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk) {
                                const uint64_t bd = desc_noswz(bb + kk * 256);
                                mma_f16(dcol, desc_sw128(ah + kk * 32), bd, idesc, (first && kk == 0) ? 0u : 1u);
                                mma_f16(dcol, desc_sw128(al + kk * 32), bd, idesc, 1u);
                            }
                        }
                        if (!ok) break;
                        mma_commit(empty_a + 8 * sa);
                        if (++sa == kNA) {
                            sa = 0;
                            pha ^= 1u;
                        }
                        mma_commit(empty_b + 8 * sb);
                        if (++sb == kNB) {
                            sb = 0;
                            phb ^= 1u;
                        }
                    }
                    if (ok && sg.commit_kb >= 0) mma_commit(acc_full + 8 * (int)(sg.commit_kb & 3));
                }
        }
    } else if (warp < 6) {
        // ------------------------------------------------------------ drawers (warps 2-5)
        // Uniform control flow: every drawer runs the whole loop nest and meets
        // every named barrier; after an abort the work is skipped.
        const int w = tid - 64;            // 0..127
        const int lane_base = 32 * (warp & 3);
        const int row = lane_base + lane;  // TMEM lane / accumulator row read in the epilogue
        const int HS = hs_stride(q), qv = q4_of(q) >> 2;  // float4s per padded row
        bool ok = true;
        long long staged = 0;  // number of correction stagings issued (by w == 0)
        if (w == 0 && nblocks > 0) {
            stage_corr(0);
            staged = 1;
        }
        for (long long kb = 0; kb < nblocks; ++kb) {
            const Blk g = blk_of(p, kb);
            const int slot = (int)(kb & 3);
            const uint64_t sweep = p.sweep0 + (uint64_t)(kb / p.nb);
            if (ok && !mbar_wait(acc_full + 8 * slot, (uint32_t)((kb >> 2) & 1), abort_flag, p.err)) ok = false;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int k = w; k < g.Bk * q; k += 128) hrow[k] = p.h[(size_t)g.i0 * q + k];
            if (ok && !mbar_wait(corr_bar, (uint32_t)(kb & 1), abort_flag, p.err)) ok = false;
            ok = !named_bar_or(1, 128, !ok || *abort_flag);  // one decision for every drawer
            // --- sequential redraw of block kb, one site at a time, one thread per chain
            const uint8_t *old = snap_of(kb);
            const uint32_t tacc = tmem + ((uint32_t)lane_base << 16) + (uint32_t)slot * p.acc_stride;
            for (int pp = 0; pp < g.Bk && ok; ++pp) {
                // accumulator rows [pp*q, pp*q + q) of the warps whose lanes hold them,
                // plus h, -> Hs[chain][a]
                const int r0 = pp * q;
                if (lane_base < r0 + q && lane_base + 32 > r0) {
                    const bool mine = row >= r0 && row < r0 + q;
                    const float hv = mine ? hrow[row] : 0.0f;
                    for (int c0 = 0; c0 < NC; c0 += 16) {
                        uint32_t v[16];
                        tmem_ld16(tacc + (uint32_t)c0, v);
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                        if (mine) {
#pragma unroll
                            for (int e = 0; e < 16; ++e) Hs[(c0 + e) * HS + (row - r0)] = hv + __uint_as_float(v[e]);
                        }
                    }
                }
                named_bar_sync(1, 128);
                const int i = g.i0 + pp;
                for (int ch = w; ch < NC; ch += 128) {
                    const uint64_t m = p.chain0 + cta0 + ch;  // global chain index
                    // the uniform first: it does not depend on the states
                    const uint32_t r24 = bm_u24(p.seed, m, sweep, (uint64_t)i, 0);
                    float H[32];
                    const float4 *hs4 = reinterpret_cast<const float4 *>(Hs + ch * HS);
#pragma unroll
                    for (int a4 = 0; a4 < 8; ++a4)
                        if (a4 < qv) {
                            const float4 t = hs4[a4];
                            H[4 * a4] = t.x;
                            H[4 * a4 + 1] = t.y;
                            H[4 * a4 + 2] = t.z;
                            H[4 * a4 + 3] = t.w;
                        }
                    // sites jj < pp of the block redrawn since the MMAs: + J_ij(., new) - J_ij(., old)
                    const float4 *cb = corr4 + (size_t)(pp * (pp - 1) / 2) * q * qv;
                    for (int jj = 0; jj < pp; ++jj) {
                        const int sn = st[ch * Sst + g.i0 + jj], so = old[ch * Ssn + jj];
                        if (sn == so) continue;
                        const float4 *rn = cb + (jj * q + sn) * qv, *ro = cb + (jj * q + so) * qv;
#pragma unroll
                        for (int a4 = 0; a4 < 8; ++a4)
                            if (a4 < qv) {
                                const float4 vn = rn[a4], vo = ro[a4];
                                H[4 * a4] += vn.x - vo.x;
                                H[4 * a4 + 1] += vn.y - vo.y;
                                H[4 * a4 + 2] += vn.z - vo.z;
                                H[4 * a4 + 3] += vn.w - vo.w;
                            }
                    }
                    float mx = -INFINITY;
#pragma unroll
                    for (int a = 0; a < 32; ++a)
                        if (a < q) {
                            H[a] *= p.beta_l2e;
                            mx = fmaxf(mx, H[a]);
                        }
                    float S = 0.0f;
#pragma unroll
                    for (int a = 0; a < 32; ++a)
                        if (a < q) {
                            S += exp2f(H[a] - mx);
                            H[a] = S;  // prefix sums of exp(beta H_a - max_b beta H_b)
                        }
                    const float thr = ((float)r24 * 5.9604644775390625e-8f) * S;
                    int pick = q - 1;
#pragma unroll
                    for (int a = 31; a >= 0; --a)
                        if (a < q && thr < H[a]) pick = a;
                    st[ch * Sst + i] = (uint8_t)pick;
                }
                named_bar_sync(1, 128);  // Hs is rewritten for the next site
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(acc_empty + 8 * slot);
            // after an odd block: snapshots of the next pair's blocks before their redraw
            if (ok && (kb & 1))
                for (long long nb2 = kb + 1; nb2 <= kb + 2 && nb2 < nblocks; ++nb2) {
                    const Blk gn = blk_of(p, nb2);
                    uint8_t *sn = snap_of(nb2);
                    for (int k = w; k < NC * gn.Bk; k += 128) {
                        const int ch = k / gn.Bk, x = k - ch * gn.Bk;
                        sn[ch * Ssn + x] = st[ch * Sst + gn.i0 + x];
                    }
                }
            named_bar_sync(1, 128);
            // the staged blocks are free again: stage the next block's
            if (w == 0 && ok && !*abort_flag && kb + 1 < nblocks) {
                stage_corr(kb + 1);
                ++staged;
            }
            if (lane == 0) mbar_arrive(ready + 8 * (int)(kb & 1));
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
        const int w = tid - 192;  // 0..127
        const bool own = w < NC;
        unsigned char *const row0 = base + lay.b + noswz_off(own ? w : 0, 0);
        const uint8_t *const strow = st + (own ? w : 0) * Sst;
        const int wrow = (own ? w : 0) * Ssn;
        int sb = 0, lap = 0;  // ring slot and lap of the current chunk
        bool ok = true;
        for (long long P = 0; P <= npairs && ok; ++P) {
            // main chunks: blocks 2P-2 and 2P-1 from their snapshots (pair slot (P-1)%2)
            int s0lo = L, s0hi = L, s1lo = L, s1hi = L;
            const uint8_t *ps0 = snap, *ps1 = snap;
            if (P >= 1) {
                const Blk g0 = blk_of(p, 2 * P - 2), g1 = blk_of(p, 2 * P - 1);
                s0lo = g0.i0;
                s0hi = g0.i0 + g0.Bk;
                s1lo = g1.i0;
                s1hi = g1.i0 + g1.Bk;
                ps0 = snap_of(2 * P - 2) + wrow;
                ps1 = snap_of(2 * P - 1) + wrow;
            }
            for (int step = 0; step < 4 && ok; ++step) {
                const Seg sg = seg_info(p, P, step);
                if (sg.n > 0 && sg.wait_kb >= 0 &&
                    !mbar_wait(ready + 8 * (int)(sg.wait_kb & 1), (uint32_t)((sg.wait_kb >> 1) & 1), abort_flag,
                               p.err)) {
                    ok = false;
                    break;
                }
                for (int k = 0; k < sg.n; ++k) {
                    if (lap > 0 && !mbar_wait(empty_b + 8 * sb, (uint32_t)((lap - 1) & 1), abort_flag, p.err)) {
                        ok = false;
                        break;
                    }
                    const int c = seg_chunk(sg, k);
                    const int k0 = c * kKC;
                    unsigned char *rowp = row0 + sb * NC * 128;
                    if (own) {
#pragma unroll
                        for (int pc = 0; pc < 8; ++pc)
                            *reinterpret_cast<uint4 *>(rowp + pc * 128) = make_uint4(0, 0, 0, 0);
                        if (!sg.delta) {
                            const int jlo = jtab[2 * c], jhi = jtab[2 * c + 1];
                            for (int j = jlo; j <= jhi; ++j) {
                                const int sj = (j >= s0lo && j < s0hi)   ? ps0[j - s0lo]
                                               : (j >= s1lo && j < s1hi) ? ps1[j - s1lo]
                                                                         : strow[j];
                                const int pos = j * q + sj - k0;
                                if (pos >= 0 && pos < kKC)
                                    *reinterpret_cast<unsigned short *>(rowp + (pos >> 3) * 128 + (pos & 7) * 2) =
                                        0x3c00u;
                            }
                        } else {
                            for (int u = 0; u < 2; ++u) {
                                const long long db = u == 0 ? sg.d0 : sg.d1;
                                if (db < 0) continue;
                                const Blk gd = blk_of(p, db);
                                const uint8_t *po = (u == 0 ? ps0 : ps1);  // d0 = 2P-2, d1 = 2P-1
                                for (int x = 0; x < gd.Bk; ++x) {
                                    const int j = gd.i0 + x;
                                    const int sn = strow[j], so = po[x];
                                    if (sn == so) continue;
                                    const int pn = j * q + sn - k0, pd = j * q + so - k0;
                                    if (pn >= 0 && pn < kKC)
                                        *reinterpret_cast<unsigned short *>(rowp + (pn >> 3) * 128 + (pn & 7) * 2) =
                                            0x3c00u;
                                    if (pd >= 0 && pd < kKC)
                                        *reinterpret_cast<unsigned short *>(rowp + (pd >> 3) * 128 + (pd & 7) * 2) =
                                            0xbc00u;
                                }
                            }
                        }
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(full_b + 8 * sb);
                    if (++sb == kNB) {
                        sb = 0;
                        ++lap;
                    }
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

// Jt[nb*128 rows][Kp/64 slabs][2 (hi, lo)][64] of T (fp16 or bf16).  Row
// blk*128 + pp*q + a holds site i = blk*B + pp, symbol a (pp < sites of the
// block; the other rows of the 128 are zero); for column k = (j,b) of slab
// k/64, hi = T(J_ij(a,b)) and lo = T(J_ij(a,b) - hi) (J_ij(a,b) = J[i][j][a][b],
// round to nearest); zero beyond L*q columns.  Each row interleaves the hi and
// lo slabs so one 3-D TMA op brings both.
__device__ __forceinline__ __half to_t(float v, __half *) { return __float2half_rn(v); }
__device__ __forceinline__ float from_t(__half v) { return __half2float(v); }
__device__ __forceinline__ __nv_bfloat16 to_t(float v, __nv_bfloat16 *) { return __float2bfloat16_rn(v); }
__device__ __forceinline__ float from_t(__nv_bfloat16 v) { return __bfloat162float(v); }

//
// fp16 holds magnitudes up to 65504.  A coupling beyond that is clamped to
// +-65504 (so the operands stay finite) and flagged in *ovf; the model's
// status call then reports BM_ENUMERIC for the tensor-core sweep.
template <typename T>
__global__ void __launch_bounds__(256) k_build_mma_layout(const float *__restrict__ J, T *__restrict__ jt, int L, int q,
                                                          int Kp, int B, int nb, int *__restrict__ ovf)
{
    // One CTA per output row r = (block, site pp of the block, symbol a);
    // thread t writes columns k = t + 256 m, whose (j, b) it advances without
    // divisions.  Row (i, a) of J is J[i][j][a][b] = src[j q^2 + b].
    constexpr bool kHalf = sizeof(T) == 2 && std::is_same<T, __half>::value;
    const int r = blockIdx.x;
    const int blk = r / kRowsA, rr = r - blk * kRowsA;
    const int pp = rr / q, a = rr - pp * q, i = blk * B + pp;
    const bool row_ok = pp < B && i < L;
    const int Q = L * q, qq = q * q;
    const float *src = J + ((size_t)(row_ok ? i : 0) * L * q + a) * q;
    T *out = jt + (size_t)r * (2 * Kp);
    const int dj = 256 / q, db = 256 - dj * q;
    int k = threadIdx.x, j = k / q, b = k - j * q;
    int bad = 0;
    for (; k < Kp; k += 256) {
        float v = 0.0f;
        if (row_ok && k < Q) v = src[(size_t)j * qq + b];
        if (kHalf && !(fabsf(v) <= 65504.0f)) {
            bad = 1;
            v = v != v ? 0.0f : copysignf(65504.0f, v);
        }
        const T vh = to_t(v, (T *)nullptr);
        const int o = ((k / kKC) * (2 * kKC)) + (k % kKC);  // slab k/64: hi then lo
        out[o] = vh;
        out[o + kKC] = to_t(v - from_t(vh), (T *)nullptr);
        b += db;
        if (b >= q) {
            b -= q;
            ++j;
        }
        j += dj;
    }
    if (bad) atomicOr(ovf, 1);
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
// 128 bytes), 128B swizzle.  box_rows x box_slabs per op: {256, 2} lands
// the hi tiles of two consecutive blocks and then their lo tiles; {128, 1}
// one tile; {128, 2} one block's hi tile and then its lo tile.
int make_map(CUtensorMap *map, const void *ptr, int rows, int Kp, int box_rows, int box_slabs,
             CUtensorMapDataType dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT16)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return bm_fail(BM_ECUDA, "cuTensorMapEncodeTiled entry point unavailable");
    cuuint64_t dims[3] = {(cuuint64_t)kKC, (cuuint64_t)rows, (cuuint64_t)(2 * Kp / kKC)};
    cuuint64_t strides[2] = {(cuuint64_t)Kp * 4, (cuuint64_t)kKC * 2};
    cuuint32_t box[3] = {(cuuint32_t)kKC, (cuuint32_t)box_rows, (cuuint32_t)box_slabs};
    cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = fn(map, dt, 3, const_cast<void *>(ptr), dims, strides, box,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return bm_fail(BM_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return BM_OK;
}

// Sites per block: as many as fill the 128 accumulator rows (at most kBmax),
// as long as the block's in-block coupling blocks (B(B-1)/2 of them, q rows
// of q rounded up to 4 floats, staged in shared memory by the sweeps) fit
// 32 KB, and at least two blocks per sweep, so that the two blocks of a pair
// never hold the same sites.  (Without the 32 KB cap, alphabets of 5 or 6
// symbols would stage 40-48 KB and leave room for too few chains per CTA.)
int block_sites(int L, int q)
{
    constexpr long long kCorrBudget = 32768;
    const long long row_bytes = (long long)q * ((q + 3) & ~3) * 4;
    int B = std::min(kBmax, kRowsA / q);
    while (B > 2 && (long long)B * (B - 1) / 2 * row_bytes > kCorrBudget) --B;
    if ((L + B - 1) / B < 2) B = (L + 1) / 2;
    return B;
}

}  // namespace

// Chains per CTA for the tensor-core sweep (multiple of 16, <= 128), or 0
// when the shape does not fit one CTA's shared memory or L < 2.
int bm_gibbs_mma_chains_per_cta(const bm_model_s *m, int M)
{
    if (m->L < 2 || m->L > 65535) return 0;  // two blocks per sweep; 16-bit site indices
    const int nsm = m->num_sms > 0 ? m->num_sms : 1;
    int nc = (M + nsm - 1) / nsm;
    nc = std::max(16, (nc + 15) & ~15);
    nc = std::min(nc, 128);  // one operand-row generator thread per chain
    const int Lp = (m->L + 15) & ~15;
    const int B = block_sites(m->L, m->q);
    const int nK = (m->L * m->q + kKC - 1) / kKC;
    while (nc >= 16 && smem_layout(nc, Lp, B, m->q, nK).total + 1024 > 227 * 1024) nc -= 16;
    return nc >= 16 ? nc : 0;
}

int bm_split_block_sites(int L, int q) { return block_sites(L, q); }

// Bring the split layout of the live J up to date: fp16 (the sweep's, maps
// tmap_j and tmap_j1) or bf16 (map tmap_bf1).
int bm_split_prepare(bm_model_s *m, int bf16, cudaStream_t st)
{
    if (bf16 ? m->bf_current : m->mma_current) return BM_OK;
    const int B = block_sites(m->L, m->q), nb = (m->L + B - 1) / B;
    const int rows = nb * kRowsA;  // every block padded to 128 rows
    const int Kp = (m->L * m->q + kKC - 1) / kKC * kKC;
    void **buf = bf16 ? &m->Jt_bf : &m->Jt;
    if (!*buf) {
        m->Kp = Kp;
        BM_CK(cudaMalloc(buf, (size_t)rows * Kp * 2 * sizeof(__half)));
        int rc;
        if (bf16) {
            rc = make_map(reinterpret_cast<CUtensorMap *>(m->tmap_bf1), *buf, rows, Kp, kRowsA, 1,
                          CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
        } else {
            rc = make_map(reinterpret_cast<CUtensorMap *>(m->tmap_j), *buf, rows, Kp, 2 * kRowsA, 2);
            if (rc == BM_OK) rc = make_map(reinterpret_cast<CUtensorMap *>(m->tmap_j1), *buf, rows, Kp, kRowsA, 1);
            if (rc == BM_OK) rc = make_map(reinterpret_cast<CUtensorMap *>(m->tmap_jp), *buf, rows, Kp, kRowsA, 2);
        }
        if (rc != BM_OK) return rc;
    }
    const int grid = rows;
    if (bf16)
        k_build_mma_layout<__nv_bfloat16><<<grid, 256, 0, st>>>(m->J, (__nv_bfloat16 *)*buf, m->L, m->q, Kp, B, nb,
                                                                 m->dflags + 5);
    else
        k_build_mma_layout<__half><<<grid, 256, 0, st>>>(m->J, (__half *)*buf, m->L, m->q, Kp, B, nb, m->dflags + 5);
    BM_CK_LAUNCH("k_build_mma_layout");
    (bf16 ? m->bf_current : m->mma_current) = true;
    return BM_OK;
}

int bm_launch_gibbs_mma(bm_model_s *m, bm_chains_s *c, int nsweeps, float beta, cudaStream_t st)
{
    const int NC = bm_gibbs_mma_chains_per_cta(m, c->M);
    if (NC == 0) return bm_fail(BM_EINVAL, "tensor-core sweep: shape does not fit shared memory");
    {
        int rc = bm_split_prepare(m, 0, st);
        if (rc == BM_OK) rc = bm_corr_prepare(m, st);
        if (rc != BM_OK) return rc;
    }
    MmaArgs a;
    a.h = m->h;
    a.Jc = m->Jc;
    a.states = c->s;
    a.err = m->dflags + 3;
    a.seed = c->seed;
    a.chain0 = c->chain0;
    a.sweep0 = c->sweep;
    a.beta_l2e = (float)((double)beta * 1.4426950408889634);
    a.M = c->M;
    a.L = c->L;
    a.q = c->q;
    a.Lp = (c->L + 15) & ~15;
    a.bs = m->bs;
    a.B = block_sites(c->L, c->q);
    a.nb = (c->L + a.B - 1) / a.B;
    a.nK = m->Kp / kKC;
    a.NC = NC;
    a.nsweeps = nsweeps;
    a.nblocks = (long long)nsweeps * a.nb;
    a.X = a.nK / 2;  // main chunks before the previous pair's first delta step
    a.acc_stride = NC <= 32 ? 32 : NC <= 64 ? 64 : 128;
    a.tmem_cols = 4 * a.acc_stride;  // four accumulators
    const Smem lay = smem_layout(NC, a.Lp, a.B, a.q, a.nK);
    const size_t smem = lay.total + 1024;
    BM_CK(cudaFuncSetAttribute(k_gibbs_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = (c->M + NC - 1) / NC;
    k_gibbs_mma<<<grid, kThreads, smem, st>>>(*reinterpret_cast<const CUtensorMap *>(m->tmap_j),
                                              *reinterpret_cast<const CUtensorMap *>(m->tmap_j1), a);
    BM_CK_LAUNCH("k_gibbs_mma");
    return BM_OK;
}
