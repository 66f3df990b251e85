// Chain pair counts as a TMA-fed product on paired tensor cores (tcgen05
// cta_group::2 + TMEM + TMA).
//
// The model statistics of Sec. 2.1 are the counts
//     C[(i,a),(j,b)] = #{m : s_i^m = a, s_j^m = b} = (X^T X)[(i,a),(j,b)],
// X the one-hot encoding of the chains, X[m][(i,a)] = [s_i^m == a].  This is
// a dense contraction over the chain index with exact 0/1 operands; FP8 E4M3
// (1.0 = 0x38) operands with FP32 accumulation give exact counts below 2^24.
//
// Two kernels:
//   k_onehot_t     writes X^T once per call: XT[(i,a)][m] (Q = L*q rows, Mp
//                  chain columns, zero padded to a multiple of 128), 16-byte
//                  stores built with four-byte SIMD compares from a
//                  shared-memory transpose of the states;
//   k_counts_pair  persistent over the output tiles that hold some pair
//                  i <= j, one CTA pair (cluster of 2) per tile at a time.  A
//                  tile is 256 rows (i,a) x 256 columns (j,b), T = floor(256/q)
//                  sites each way.  CTA r holds rows [128r, 128r+128) of the
//                  tile's A operand and of its B operand (the B half that the
//                  paired MMA reads from that CTA); per stage of 128 chains
//                  each CTA's warp 0 loads its two 16 KB halves by TMA (3-D
//                  view, 128B swizzle) into a 6-stage ring, the completions
//                  counted on CTA 0's barrier.  CTA 0's warp 1 issues 4 paired
//                  MMAs per stage (kind::f8f6f4, M = 256, N = 256, K = 32);
//                  each CTA's TMEM receives its 128 rows x 256 columns.  Two
//                  accumulator buffers (2 x 256 columns) let the epilogue of
//                  one tile run while the next one accumulates.  Warps 2-9 of
//                  each CTA (two groups of four, one per 128-column half)
//                  store the int32 counts of the blocks i <= j in the upper
//                  block-triangle layout.
//                  Schedule: each pair takes nfull = ntiles / npairs whole
//                  tiles; the R = ntiles mod npairs remaining tiles are split
//                  into s parts along the chains, one part per pair, taken
//                  first, so every pair ends after about ntiles / npairs
//                  tiles.  A part's epilogue writes its int32 partial counts
//                  to a workspace, releases its accumulator and takes a
//                  ticket (device-scope CAS after a fence; the ticket word
//                  carries the launch's epoch, so a ticket left by an earlier
//                  launch counts as none); the part that draws the last
//                  ticket sums all the partials from the workspace and stores
//                  them while its pair's next tile accumulates.  No part waits
//                  on another, and the sums are exact in any order.
// Every mbarrier wait is bounded by %globaltimer (2 s); a timeout sets the
// chains' device error word (bit 2), every role leaves its loop and TMEM is
// released.
#include "bm_internal.cuh"
#include "tc_common.cuh"

#include <cuda.h>

#include <algorithm>
#include <mutex>

namespace {

using namespace bmtc;

constexpr int kTile = 256;            // output tile: 256 rows (i,a) x 256 columns (j,b)
constexpr int kHalf = 128;            // rows of the tile held by each CTA of the pair
constexpr int kKB = 128;              // chains per stage (one 128-byte swizzle atom per row)
constexpr int kStageA = kHalf * kKB;  // 16 KB: this CTA's A rows
constexpr int kStageB = kHalf * kKB;  // 16 KB: this CTA's B rows
constexpr int kNS = 6;                // stages
constexpr int kThreads = 320;         // 10 warps: producer, MMA issuer, 8 epilogue warps
constexpr int kSlab = 16;             // accumulator columns staged per epilogue pass
constexpr int kStgStride = 17;        // staging row stride (int32): conflict-free copy-in
constexpr int kGroupCols = 128;       // columns of the tile per epilogue group
constexpr int kMaxParts = 4;          // parts per split tile (the last part reads the others)
constexpr int kUnitInts = kHalf * kGroupCols;  // partial counts of one CTA's epilogue group

// ---------------------------------------------------------------------------
// X^T, E4M3 one-hot.  Block: 128 chains x 32 sites, 256 threads.
// ---------------------------------------------------------------------------
constexpr int kOtChains = 128, kOtSites = 32;

__global__ void __launch_bounds__(256) k_onehot_t(const uint8_t *__restrict__ S, int M, int L, int q, int Mp,
                                                  uint8_t *__restrict__ XT)
{
    __shared__ __align__(16) uint8_t sv[kOtSites][kOtChains + 16];  // states transposed: [site][chain]
    const int m0 = blockIdx.x * kOtChains, i0 = blockIdx.y * kOtSites;
    const int ns = min(kOtSites, L - i0);
    // all loads of a thread in flight before the first shared-memory store
    constexpr int kPer = kOtChains * kOtSites / 256;
    uint8_t ld[kPer];
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        const int k = threadIdx.x + 256 * u;
        const int c = k / kOtSites, x = k - c * kOtSites;  // consecutive threads: consecutive sites of a chain
        const int m = m0 + c;
        ld[u] = (m < M && x < ns) ? S[(size_t)m * L + i0 + x] : (uint8_t)0xff;  // 0xff: padding chain
    }
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        const int k = threadIdx.x + 256 * u;
        sv[k % kOtSites][k / kOtSites] = ld[u];
    }
    __syncthreads();
    // rows (i,a) of this site range, 8 segments of 16 chains each; a byte of
    // the row is 0x38 where the chain's state equals a
    const int nrow = ns * q;
#pragma unroll 4
    for (int k = threadIdx.x; k < nrow * 8; k += blockDim.x) {
        const int r = k >> 3, seg = k & 7;
        const int x = r / q, a = r - x * q;
        const uint4 st4 = *reinterpret_cast<const uint4 *>(&sv[x][seg * 16]);
        const unsigned int aa = (unsigned int)a * 0x01010101u;
        const uint4 w = make_uint4(__vcmpeq4(st4.x, aa) & 0x38383838u, __vcmpeq4(st4.y, aa) & 0x38383838u,
                                   __vcmpeq4(st4.z, aa) & 0x38383838u, __vcmpeq4(st4.w, aa) & 0x38383838u);
        const size_t row = (size_t)(i0 + x) * q + a;
        *reinterpret_cast<uint4 *>(XT + row * Mp + m0 + seg * 16) = w;
    }
}

// ---------------------------------------------------------------------------
// Persistent counts product on CTA pairs.
// ---------------------------------------------------------------------------
struct CtArgs {
    int32_t *counts;
    int *err;
    int32_t *ws;  // [R*s][2 CTAs][2 groups][kHalf][kGroupCols] partial counts of the split tiles
    unsigned long long *cnt;  // [R][2][2] arrival tickets: launch epoch (high word), arrivals (low word)
    unsigned int epoch;       // this launch's epoch (never 0)
    int L, q, TI, TJ, nti, ntj, ntiles, nstages;  // nstages: K stages (128 chains each) per tile
    int npairs, nfull, R, s;                      // schedule (see the file comment)
};

// Work unit n of pair cl: a whole tile (part < 0) or part `part` of a split
// tile, covering K stages [k0, k1).  Returns false past the pair's last unit.
struct Unit {
    int t, part, tr, k0, k1;
};

__device__ __forceinline__ bool unit_of(const CtArgs &p, int cl, int n, Unit &u)
{
    // The pairs cl < R*s start with their part of a split tile, so that its
    // partial write, ticket and combine overlap the whole tiles' MMAs.
    const bool has_part = cl < p.R * p.s;
    if (has_part && n == 0) {
        u.tr = cl % p.R;
        u.t = p.nfull * p.npairs + u.tr;
        if (p.s == 1) {
            u.part = -1;
            u.k0 = 0;
            u.k1 = p.nstages;
        } else {
            u.part = cl / p.R;
            u.k0 = (int)((long long)u.part * p.nstages / p.s);
            u.k1 = (int)((long long)(u.part + 1) * p.nstages / p.s);
        }
        return true;
    }
    const int f = n - (has_part ? 1 : 0);  // whole tile index of this pair
    if (f >= p.nfull) return false;
    u.t = cl + f * p.npairs;
    u.part = -1;
    u.tr = -1;
    u.k0 = 0;
    u.k1 = p.nstages;
    return true;
}

// Tile t of the list of tiles holding some pair i <= j, in row-tile-major
// order: row tile ti holds sites [ti*TI, ...), column tile tj sites
// [tj*TJ, ...); tile (ti, tj) is needed when its last column site >= its
// first row site.
__device__ __forceinline__ void tile_of(const CtArgs &p, int t, int &ti, int &tj)
{
    // column tiles needed for row tile ti: tj >= tj0(ti) = floor(ti*TI / TJ)
    int acc = 0;
    for (ti = 0; ti < p.nti; ++ti) {
        const int tj0 = (ti * p.TI) / p.TJ;
        const int n = p.ntj - tj0;
        if (t < acc + n) {
            tj = tj0 + (t - acc);
            return;
        }
        acc += n;
    }
    tj = 0;
}

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t leader_addr(uint32_t a)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, 0;" : "=r"(r) : "r"(a));
    return r;
}

__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void mma_f8_pair(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// Arrive once on the barrier at shared offset `bar` of both CTAs of the pair
// when every MMA issued so far by this thread has completed.
__device__ __forceinline__ void mma_commit_pair(uint32_t bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(bar),
        "h"((uint16_t)3)
        : "memory");
}

__device__ __forceinline__ void mbar_arrive_cluster(uint32_t a)
{
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(a) : "memory");
}

__device__ __forceinline__ bool mbar_wait_cluster(uint32_t bar, uint32_t parity, volatile int *abort_flag, int *err)
{
    const uint64_t t0 = gtimer();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity), "r"(kSuspendNs)
            : "memory");
        if (ok) return true;
        if (*abort_flag) return false;
        if (gtimer() - t0 > kWaitNs) {
            *abort_flag = 1;
            atomicOr(err, 4);
            return false;
        }
    }
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
    k_counts_pair(const __grid_constant__ CUtensorMap tm_x, const CtArgs p)
{
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = su32(smem_raw);
    unsigned char *base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    // stage s: A (this CTA's 128 rows) at s*(kStageA + kStageB), B right after;
    // then per epilogue group its staging of one 16-column slab, and the tickets
    int32_t *stg = reinterpret_cast<int32_t *>(base + kNS * (kStageA + kStageB));  // [2][kHalf][kStgStride]
    volatile int *ticket = stg + 2 * kHalf * kStgStride;                                 // [2]
    uint64_t *bars = reinterpret_cast<uint64_t *>(stg + 2 * kHalf * kStgStride + 2);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * kNS + 5);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const uint32_t full = su32(bars), empty = full + 8 * kNS;
    const uint32_t acc_full = empty + 8 * kNS, acc_empty = acc_full + 16;  // two each (accumulator buffers)
    const uint32_t fin = acc_empty + 16;  // completion of every MMA issued (teardown)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = p.q, L = p.L;
    const int r = (int)cluster_rank();
    const int cl = blockIdx.x >> 1;

    if (tid == 0) {
        for (int s = 0; s < kNS; ++s) {
            mbar_init(full + 8 * s, 1);
            mbar_init(empty + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(acc_full + 8 * b, 1);
            mbar_init(acc_empty + 8 * b, 16);  // 8 epilogue warps of each CTA
        }
        mbar_init(fin, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {  // one warp of each CTA of the pair; both get the same columns
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(2 * kTile)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    cluster_sync();  // both CTAs' barriers are initialised before any copy or arrival reaches them
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer (both CTAs)
        if (lane == 0) {
            int s = 0, lap = 0;
            long long issued = 0;
            bool ok = true;
            Unit u;
            for (int n = 0; ok && unit_of(p, cl, n, u); ++n) {
                int ti, tj;
                tile_of(p, u.t, ti, tj);
                const int ya = ti * p.TI * q + kHalf * r, yb = tj * p.TJ * q + kHalf * r;
                for (int k = u.k0; k < u.k1; ++k) {
                    if (lap > 0 && !mbar_wait(empty + 8 * s, (uint32_t)((lap - 1) & 1), abort_flag, p.err)) {
                        ok = false;
                        break;
                    }
                    const uint32_t dst = su32(base + s * (kStageA + kStageB));
                    const uint32_t fb = leader_addr(full + 8 * s);
                    if (r == 0) mbar_expect_tx(full + 8 * s, 2 * (kStageA + kStageB));  // both CTAs' bytes
                    tma_load_3d_cg2(dst, &tm_x, 0, ya, k, fb);
                    tma_load_3d_cg2(dst + kStageA, &tm_x, 0, yb, k, fb);
                    ++issued;
                    if (++s == kNS) {
                        s = 0;
                        ++lap;
                    }
                }
            }
            if (*abort_flag) {  // let the copies in flight land before exit
                if (r == 0) {
                    volatile int no_abort = 0;
                    for (long long u = issued > kNS ? issued - kNS : 0; u < issued; ++u)
                        mbar_wait(full + 8 * (int)(u % kNS), (uint32_t)((u / kNS) & 1), &no_abort, p.err);
                } else {
                    __nanosleep(100000);  // this CTA's completions are counted on CTA 0's barriers
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer (CTA 0)
        if (r == 0 && lane == 0) {
            // kind::f8f6f4: D F32 (bit 4), A = B = E4M3 (0), K-major, N >> 3 at 17, M >> 4 at 24.
            const uint32_t idesc = (1u << 4) | ((uint32_t)(kTile >> 3) << 17) | ((uint32_t)(kTile >> 4) << 24);
            int s = 0;
            uint32_t ph = 0;
            bool ok = true;
            Unit u;
            for (int n = 0; ok && unit_of(p, cl, n, u); ++n) {
                const int b = n & 1;
                if (n >= 2 && !mbar_wait_cluster(acc_empty + 8 * b, (uint32_t)(((n - 2) >> 1) & 1), abort_flag, p.err)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + (uint32_t)(b * kTile);
                for (int k = u.k0; k < u.k1; ++k) {
                    if (!mbar_wait(full + 8 * s, ph, abort_flag, p.err)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t a0 = su32(base + s * (kStageA + kStageB)), b0 = a0 + kStageA;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        mma_f8_pair(d, desc_sw128(a0 + kk * 32), desc_sw128(b0 + kk * 32), idesc,
                                    (k > u.k0 || kk > 0) ? 1u : 0u);
                    mma_commit_pair(empty + 8 * s);
                    if (++s == kNS) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
                if (!ok) break;
                mma_commit_pair(acc_full + 8 * b);
            }
            // all MMAs of this thread retired before TMEM is released (also after an abort)
            mma_commit_pair(fin);
            volatile int no_abort = 0;
            mbar_wait(fin, 0, &no_abort, p.err);
        }
    } else {
        // ------------------------------------------------------------ epilogue (warps 2-9, both CTAs)
        // Group g (warps 2-5 or 6-9) handles columns [128g, 128g + 128) of the
        // tile's rows held by this CTA.  Per 16-column slab: each warp copies
        // its 32 accumulator rows to the group's staging buffer (one row per
        // lane), then the group's 128 threads write the slab out, 16
        // consecutive columns per half-warp, so a store covers a contiguous
        // run of a block row.  The output offset of (row, column) splits into
        // a row term and a column term,
        //   ((i*L - i(i-1)/2 - i) q^2 + a q) + (j q^2 + b),
        // and the pair (i, j) is stored when i <= j; a thread's 16 rows are
        // the same in every slab, so their terms are computed once per tile.
        // A part of a split tile writes its partial counts to the workspace,
        // releases its accumulator and takes a ticket; the last part sums the
        // partials from the workspace and stores them while the pair's next
        // tile accumulates.  Uniform control flow within the group (its named
        // barrier) also after an abort.
        constexpr int kRowsPerThread = kHalf / (128 / kSlab);  // 16
        constexpr int kPieces = kSlab / 4;                     // 16-byte pieces of a row's slab
        const int g = (warp - 2) >> 2;
        const int quarter = warp & 3;                 // TMEM lane quarter this warp may read
        const int lr = 32 * quarter + lane;           // local row copied by this thread
        const int e = tid - 64 - 128 * g;             // 0..127 within the group
        const int ce = e & (kSlab - 1);
        const int bar_id = 1 + g;
        int32_t *gst = stg + g * kHalf * kStgStride;
        const long long q2 = (long long)q * q;
        const uint32_t acc_empty_leader = leader_addr(acc_empty);
        bool ok = true;
        Unit u;
        for (int n = 0; unit_of(p, cl, n, u); ++n) {
            const int b = n & 1;
            int ti, tj;
            tile_of(p, u.t, ti, tj);
            long long rt[kRowsPerThread];  // row terms of rows e/16 + 8k
            int rs[kRowsPerThread];        // their sites (INT_MAX: padding row)
#pragma unroll
            for (int k = 0; k < kRowsPerThread; ++k) {
                const int R = kHalf * r + (e >> 4) + 8 * k;  // tile row
                const int il = R / q, a = R - il * q;
                const int i = ti * p.TI + il;
                const bool valid = il < p.TI && i < L;
                rs[k] = valid ? i : 0x7fffffff;
                rt[k] = valid ? ((long long)i * L - (long long)i * (i - 1) / 2 - i) * q2 + (long long)a * q : 0;
            }
            if (ok && !mbar_wait(acc_full + 8 * b, (uint32_t)((n >> 1) & 1), abort_flag, p.err)) ok = false;
            if (named_bar_or(bar_id, 128, !ok || *abort_flag)) {  // the same decision in every thread of the group
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t tacc = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(b * kTile + g * kGroupCols);
            const int ci = (u.tr * 2 + r) * 2 + g;  // ticket of this CTA half and group of the split tile
            // A part's partial counts: [slab][piece][local row] 16-byte pieces,
            // so a warp writes or reads 512 contiguous bytes per instruction.
            auto unit_ws = [&](int part, int c0) {
                return reinterpret_cast<int4 *>(p.ws + (size_t)((u.tr * p.s + part) * 4 + r * 2 + g) * kUnitInts) +
                       (size_t)(c0 / kSlab) * kPieces * kHalf + lr;
            };
            // Write-out of one staged 16-column slab: thread e handles column
            // c0 + (e & 15) of rows e/16 + 8k.
            auto store_slab = [&](int c0) {
                const int cc = g * kGroupCols + c0 + ce;
                const int jl = cc / q, bb = cc - jl * q;
                const int j = tj * p.TJ + jl;
                const int csite = (jl < p.TJ && j < L) ? j : -1;
                const long long cterm = (long long)j * q2 + bb;
                int32_t val[kRowsPerThread];
#pragma unroll
                for (int k = 0; k < kRowsPerThread; ++k) val[k] = gst[((e >> 4) + 8 * k) * kStgStride + ce];
#pragma unroll
                for (int k = 0; k < kRowsPerThread; ++k)
                    if (rs[k] <= csite) p.counts[rt[k] + cterm] = val[k];
            };
            auto stage = [&](const int32_t (&x16)[kSlab]) {
#pragma unroll
                for (int x = 0; x < kSlab; ++x) gst[lr * kStgStride + x] = x16[x];
            };
            if (u.part < 0) {  // a whole tile: store the counts from the accumulator
                for (int c0 = 0; c0 < kGroupCols; c0 += kSlab) {
                    uint32_t v[kSlab];
                    tmem_ld16(tacc + (uint32_t)c0, v);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    int32_t x16[kSlab];
#pragma unroll
                    for (int x = 0; x < kSlab; ++x) x16[x] = (int32_t)__uint_as_float(v[x]);
                    stage(x16);
                    named_bar_sync(bar_id, 128);
                    store_slab(c0);
                    named_bar_sync(bar_id, 128);  // staging is rewritten by the next slab
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive_cluster(acc_empty_leader + 8 * b);
            } else {
                // a part of a split tile: write the partial, release the
                // accumulator, take a ticket; the last part sums all partials
                for (int c0 = 0; c0 < kGroupCols; c0 += kSlab) {
                    uint32_t v[kSlab];
                    tmem_ld16(tacc + (uint32_t)c0, v);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    int4 *dst = unit_ws(u.part, c0);
#pragma unroll
                    for (int x = 0; x < kPieces; ++x)
                        __stcg(dst + (size_t)x * kHalf,
                               make_int4((int)__uint_as_float(v[4 * x]), (int)__uint_as_float(v[4 * x + 1]),
                                         (int)__uint_as_float(v[4 * x + 2]), (int)__uint_as_float(v[4 * x + 3])));
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive_cluster(acc_empty_leader + 8 * b);
                named_bar_sync(bar_id, 128);
                if (e == 0) {
                    __threadfence();  // this group's partial is visible device-wide before its ticket
                    // arrivals of this launch; a ticket left by an earlier
                    // launch (other epoch) counts as none
                    unsigned long long *cw = p.cnt + ci;
                    unsigned long long old = *reinterpret_cast<volatile unsigned long long *>(cw), nw = 0;
                    int tk = -1;
                    for (int it = 0; it < (1 << 16); ++it) {  // a failed swap means another part's arrival landed
                        nw = (unsigned int)(old >> 32) == p.epoch ? old + 1ull
                                                                   : (((unsigned long long)p.epoch << 32) | 1ull);
                        const unsigned long long seen = atomicCAS(cw, old, nw);
                        if (seen == old) {
                            tk = (int)(unsigned int)nw;
                            break;
                        }
                        old = seen;
                    }
                    if (tk < 0) atomicOr(p.err, 4);
                    __threadfence();
                    ticket[g] = tk;
                }
                named_bar_sync(bar_id, 128);
                if (ticket[g] == p.s) {  // the s-th arrival: every partial is in the workspace
                    // the partials of slab c0 + 16 are loaded while slab c0 is stored
                    int4 nxt[kMaxParts][kPieces];
                    auto load = [&](int c0) {
#pragma unroll
                        for (int pp = 0; pp < kMaxParts; ++pp)
#pragma unroll
                            for (int x = 0; x < kPieces; ++x)
                                nxt[pp][x] = pp < p.s ? __ldcg(unit_ws(pp, c0) + (size_t)x * kHalf) : make_int4(0, 0, 0, 0);
                    };
                    load(0);
                    for (int c0 = 0; c0 < kGroupCols; c0 += kSlab) {
                        int32_t x16[kSlab];
#pragma unroll
                        for (int x = 0; x < kPieces; ++x) {
                            int4 t4 = nxt[0][x];
#pragma unroll
                            for (int pp = 1; pp < kMaxParts; ++pp) {
                                t4.x += nxt[pp][x].x;
                                t4.y += nxt[pp][x].y;
                                t4.z += nxt[pp][x].z;
                                t4.w += nxt[pp][x].w;
                            }
                            x16[4 * x] = t4.x;
                            x16[4 * x + 1] = t4.y;
                            x16[4 * x + 2] = t4.z;
                            x16[4 * x + 3] = t4.w;
                        }
                        if (c0 + kSlab < kGroupCols) load(c0 + kSlab);
                        stage(x16);
                        named_bar_sync(bar_id, 128);
                        store_slab(c0);
                        named_bar_sync(bar_id, 128);
                    }
                }
            }
        }
        if (!ok) *abort_flag = 1;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // CTA 0's MMAs have retired (its issuer waited on `fin`); no arrival or
    // copy is headed for either CTA past this barrier
    cluster_sync();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kTile) : "memory");
    cluster_sync();
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
        cudaDriverEntryPointQueryResult qr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &qr) ==
                cudaSuccess &&
            qr == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(f);
    });
    return fn;
}

// 3-D view of XT [Q rows][Mp bytes]: dim 0 = 128 chains of an atom
// (contiguous), dim 1 = row (stride Mp), dim 2 = atom index (stride 128);
// box {128, rows, 1}: one 128-chain atom of `rows` rows.
int make_xt_map(CUtensorMap *map, const uint8_t *xt, int Q, int Mp, int rows)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return bm_fail(BM_ECUDA, "cuTensorMapEncodeTiled entry point unavailable");
    cuuint64_t dims[3] = {(cuuint64_t)kKB, (cuuint64_t)Q, (cuuint64_t)(Mp / kKB)};
    cuuint64_t strides[2] = {(cuuint64_t)Mp, (cuuint64_t)kKB};
    cuuint32_t box[3] = {(cuuint32_t)kKB, (cuuint32_t)rows, 1u};
    cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<uint8_t *>(xt), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return bm_fail(BM_ECUDA, "cuTensorMapEncodeTiled (one-hot) failed (%d)", (int)r);
    return BM_OK;
}

}  // namespace

int bm_launch_chain_stats_tc(bm_chains_s *c, int32_t *counts, cudaStream_t st)
{
    const int M = c->M, L = c->L, q = c->q;
    if (M >= (1 << 24)) return bm_fail(BM_EINVAL, "chain_stats (tensor cores): M >= 2^24 not exact in FP32");
    const int Q = L * q;
    const int Mp = (M + kKB - 1) / kKB * kKB;  // chains zero padded to whole 128-chain stages
    const size_t bytes = (size_t)Q * Mp;
    if (!c->xt || c->xt_rows != Q || c->xt_cols != Mp) {
        if (c->xt) cudaFree(c->xt);
        c->xt = nullptr;
        BM_CK(cudaMalloc(&c->xt, bytes));
        c->xt_rows = Q;
        c->xt_cols = Mp;
        const int rc = make_xt_map(reinterpret_cast<CUtensorMap *>(c->tmap_a), (const uint8_t *)c->xt, Q, Mp, kHalf);
        if (rc != BM_OK) return rc;
    }
    dim3 g1((Mp + kOtChains - 1) / kOtChains, (L + kOtSites - 1) / kOtSites);
    k_onehot_t<<<g1, 256, 0, st>>>(c->s, M, L, q, Mp, (uint8_t *)c->xt);
    BM_CK_LAUNCH("k_onehot_t");

    CtArgs a;
    a.counts = counts;
    a.err = c->derr;
    a.L = L;
    a.q = q;
    a.TI = kTile / q;
    a.TJ = kTile / q;
    a.nti = (L + a.TI - 1) / a.TI;
    a.ntj = (L + a.TJ - 1) / a.TJ;
    a.ntiles = 0;
    for (int ti = 0; ti < a.nti; ++ti) a.ntiles += a.ntj - (ti * a.TI) / a.TJ;
    a.nstages = Mp / kKB;
    int dev = 0, nsm = 0;
    BM_CK(cudaGetDevice(&dev));
    BM_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int maxpairs = std::max(1, nsm / 2);
    a.npairs = maxpairs;
    a.nfull = a.ntiles / maxpairs;
    a.R = a.ntiles % maxpairs;
    a.s = a.R ? std::max(1, std::min(std::min(maxpairs / a.R, kMaxParts), a.nstages)) : 0;
    const int pairs = a.nfull > 0 ? maxpairs : a.R * a.s;
    if (a.s > 1 && (!c->ct_ws || !c->ct_cnt)) {  // sized for any schedule of this device: R*s <= maxpairs
        if (!c->ct_ws) BM_CK(cudaMalloc(&c->ct_ws, (size_t)maxpairs * 4 * kUnitInts * sizeof(int32_t)));
        if (!c->ct_cnt) {
            BM_CK(cudaMalloc(&c->ct_cnt, (size_t)maxpairs * 4 * sizeof(unsigned long long)));
            BM_CK(cudaMemsetAsync(c->ct_cnt, 0, (size_t)maxpairs * 4 * sizeof(unsigned long long), st));
        }
    }
    a.ws = c->ct_ws;
    a.cnt = c->ct_cnt;
    if (++c->ct_epoch == 0) c->ct_epoch = 1;  // epoch 0 marks a ticket never taken
    a.epoch = c->ct_epoch;
    const size_t smem = (size_t)kNS * (kStageA + kStageB) + ((size_t)2 * kHalf * kStgStride + 2) * 4 +
                        (2 * kNS + 5) * 8 + 16 + 1024;
    BM_CK(cudaFuncSetAttribute(k_counts_pair, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_counts_pair<<<2 * pairs, kThreads, smem, st>>>(*reinterpret_cast<const CUtensorMap *>(c->tmap_a), a);
    BM_CK_LAUNCH("k_counts_pair");
    return BM_OK;
}
