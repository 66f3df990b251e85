// Persistent-chain Gibbs sweeps on the 5th-generation tensor cores, split
// over the two CTAs of a thread-block cluster.
//
// Method: Sec. 2.1 ("Monte Carlo estimation of the gradient"), sweep = every
// site once in order (Sec. 3.3).  The arithmetic is that of the single-CTA
// tensor-core sweep (k_gibbs_mma.cu): sites in blocks of B <= floor(128/q)
// (bm_split_block_sites), the fields of a block's 128 rows (i,a) as the
// contraction of the coupling
// rows (fp16 hi + fp16 lo, FP32 accumulation in TMEM) with the one-hot
// states, then an exact sequential redraw of the block's sites with in-block
// corrections, blocks taken in pairs (2P, 2P+1).
//
// Split.  Both CTAs of a cluster hold the same NC chains, each a full copy of
// their states in its shared memory.  CTA r owns the blocks 2P + r: it loads
// only their coupling rows (one 32 KB TMA op per 64-column K chunk: the hi
// and lo tiles of 128 rows), accumulates only their fields and redraws only
// them.  Compared with one CTA doing both blocks of a pair for NC/2 chains,
// each SM moves half the coupling bytes per chunk through shared memory and
// its MMAs are twice as wide (N = NC), so the shared-memory bandwidth that
// bounds the single-CTA form buys about twice the MMA work per byte.
//
// Exchange.  After redrawing a block each drawer thread copies its chain's
// new states of the block into the peer's copy (st.shared::cluster) and
// arrives on the peer's ready barrier of that block's parity with release
// semantics at cluster scope; waiters acquire at cluster scope.  CTA 0 makes
// that copy of block 2P only once CTA 1's generators have finished pair P's
// main chunks (gen_done), which read block 2P's pre-redraw states.
// Schedule of pair P in CTA r, each step a run of 64-column K chunks:
//   A  main chunks [0, X) into block 2P+r: states after block 2P-3, with
//      blocks 2P-2 and 2P-1 (being redrawn) from their pre-redraw snapshots;
//   B  (CTA 1 only) delta chunks of block 2P-2 (+1 at the new, -1 at the old
//      state of each changed site) into block 2P-1, once block 2P-2's states
//      arrived from CTA 0; this completes block 2P-1;
//   C  main chunks [X, nK) into block 2P+r;
//   D  delta chunks of blocks 2P-2 and 2P-1 into block 2P+r; this completes
//      block 2P in CTA 0 (block 2P+1 is completed by step B of pair P+1).
// Snapshots (a block's states before its redraw; used for the blocks being
// redrawn during the main chunks, for the delta chunks and for the in-block
// corrections) of pair (2P+2, 2P+3) are taken in each CTA while no CTA can
// be writing those sites: in CTA 1 right after it redrew block 2P+1 and
// before it publishes it; in CTA 0 once block 2P+1 has arrived and before
// CTA 0 redraws block 2P+2 (its generator waits for them at step D).
//
// Data path per CTA (one CTA per SM, NC <= 160 chains, NC a multiple of 16):
//   warp 0       TMA producer (3-slot ring of 32 KB coupling tiles);
//   warp 1       TMEM allocation (two accumulators of NC columns, own block
//                j = kb/2 in slot j % 2) and the single MMA-issuing thread
//                (M = 128 rows, N = NC chains, K = 16, hi and lo);
//   warps 2-6    drawers, one thread per chain: warps 2-5 read the four TMEM
//                lane quarters of a site's rows, add h and store them as one
//                padded row per chain; each thread reads its row and the
//                staged in-block coupling blocks (padded layout Jc, one bulk
//                copy per block) with 128-bit loads, then draws (draw_symbol;
//                the block's Philox numerators are computed while its
//                accumulator fills);
//   warps 7-11   generators of the one-hot operand tiles (2-slot ring), one
//                thread per chain (zero the row, then store its few nonzeros).
// Every wait is bounded by %globaltimer (2 s); a timeout sets the CTA's abort
// flag and bit 2 of the model's device error word.  Both CTAs meet at a
// cluster barrier before leaving, and the chains are written back only when
// neither CTA aborted.
//
// Batch mode (k_gibbs_pair<true, QC>): cluster k runs work item k of a list,
// i.e. its own model's arguments, TMA descriptor and chain tile, so many
// models of uneven length are swept in one launch.
#include "bm_internal.cuh"
#include "tc_common.cuh"

#include <cuda.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

using namespace bmtc;

namespace {

constexpr int kNA = 3;                  // coupling ring slots
constexpr int kNB = 2;                  // one-hot ring slots (NC x 128 bytes each)
constexpr int kNB2 = 3;                 // the same with paired tensor cores (NC/2 x 128 bytes each)
static_assert(kNB <= kNA && kNB2 <= kNA, "one-hot slots are freed through the coupling ring's barriers");
constexpr int kKC = 64;                 // fp16 K elements per chunk (128-byte rows)
constexpr int kRowsA = 128;             // MMA M
constexpr int kTileA = kRowsA * 128;    // one hi or lo tile (16 KB)
constexpr int kSlotA = 2 * kTileA;      // ring slot: hi tile, then lo tile
constexpr int kQmax = 32;
constexpr int kBmax = 32;
constexpr int kDrawWarps = 5, kGenWarps = 5;
constexpr int kDraw = 32 * kDrawWarps;  // drawer threads
constexpr int kGen = 32 * kGenWarps;    // generator threads
constexpr int kThreads = 64 + kDraw + kGen;
constexpr int kNCmax = 160;
constexpr int kNBars = 2 * kNA + 2 * kNB2 + 2 + 2 + 2 + 1 + 1 + 1 + kNA + 1;

// ---------------------------------------------------------------- cluster helpers
__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t peer_addr(uint32_t a, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}

__device__ __forceinline__ void st_cluster_u8(uint32_t a, unsigned short v)
{
    asm volatile("st.shared::cluster.u8 [%0], %1;" ::"r"(a), "h"(v) : "memory");
}

__device__ __forceinline__ uint32_t ld_cluster_u32(uint32_t a)
{
    uint32_t v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}

__device__ __forceinline__ void mbar_arrive_peer(uint32_t a)
{
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(a) : "memory");
}

// Remote arrival without release semantics (about 10x cheaper for the issuing
// thread).  Used only to relay a completion the thread has already observed
// on its own CTA's barrier (TMA bytes landed; generator stores fenced for the
// async proxy and arrived with release), so the relayed data is in place.
__device__ __forceinline__ void mbar_arrive_peer_relaxed(uint32_t a)
{
    asm volatile("mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [%0];" ::"r"(a) : "memory");
}

__device__ __forceinline__ bool mbar_try_cl(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_try_cl_suspend(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(kSuspendNs)
        : "memory");
    return ok != 0;
}

// Bounded wait with acquire semantics at cluster scope (barriers that the
// peer CTA arrives on, or whose arrivals follow data the peer wrote); the
// waiting thread is suspended between probes, as in mbar_wait.
__device__ __forceinline__ bool mbar_wait_cl(uint32_t bar, uint32_t parity, volatile int *abort_flag, int *err)
{
    if (mbar_try_cl(bar, parity)) return true;
    const uint64_t t0 = gtimer();
    for (;;) {
        if (mbar_try_cl_suspend(bar, parity)) return true;
        if (*abort_flag) return false;
        if (gtimer() - t0 > kWaitNs) {
            *abort_flag = 1;
            atomicOr(err, 4);
            return false;
        }
    }
}

__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

struct PairArgs {
    const float *h;
    const float *Jc;  // in-block coupling blocks: [site block][pair slot][b][a padded to q4]
    uint8_t *states;
    int *err;
    uint64_t seed, sweep0, chain0;
    float beta_l2e;   // beta * log2(e): weights exp(beta H) = 2^(beta log2(e) H)
    int M, L, q, Lp, B, nb, nK, X, NC;
    int na, nmma;     // tensor-memory operand form: coupling ring slots, MMA N (block rows rounded up to 16)
    int sampler;      // BM_SAMPLER_GIBBS or BM_SAMPLER_METROPOLIS
    long long nblocks;
    uint32_t tmem_cols, acc_stride;
};

// One cluster's work in a batch of models: the model's arguments, its
// coupling tensor map (a TMA descriptor in device memory; the struct takes
// CUtensorMap's alignment) and the first chain of the cluster's tile.
struct PairItem {
    CUtensorMap tm;
    PairArgs a;
    long long first;
};

__host__ __device__ inline int st_stride(int Lp) { return Lp + 4; }
__host__ __device__ inline int snap_stride(int B) { return 4 * (((B + 3) / 4) | 1); }
__host__ __device__ inline int q4_of(int q) { return (q + 3) & ~3; }
// Row stride (floats) of the staged fields, one row per chain: q rounded up
// to 4, plus 4 when that is an even number of 16-byte units, so that eight
// consecutive rows start in eight different 16-byte bank groups.
__host__ __device__ inline int hs_stride(int q) { return ((q4_of(q) >> 2) & 1) ? q4_of(q) : q4_of(q) + 4; }
__host__ __device__ inline int corr_slots(int B) { return B * (B - 1) / 2; }

struct Smem {
    uint32_t a, b, hs, st, snap, corr, hrow, jtab, bars, misc, total;
};

// nrows_b: one-hot operand rows per CTA (NC, or NC/2 when the two CTAs'
// tensor cores are paired and each holds half of the chains' rows).
__host__ __device__ inline Smem smem_layout(int NC, int Lp, int B, int nK, int q, int nrows_b)
{
    Smem s;
    s.a = 0;
    s.b = s.a + kNA * kSlotA;
    s.hs = s.b + (nrows_b < NC ? kNB2 : kNB) * nrows_b * 128;
    s.st = s.hs + NC * hs_stride(q) * 4;          // fields h + G of one site: [chain][a]
    s.snap = s.st + NC * st_stride(Lp);           // [2 pair slots][2 blocks][NC][snap_stride]
    s.corr = (s.snap + 4 * NC * snap_stride(B) + 15) & ~15u;
    s.hrow = s.corr + (uint32_t)corr_slots(B) * q * q4_of(q) * 4;
    s.jtab = s.hrow + kRowsA * 4;
    s.bars = (s.jtab + nK * 8 + 15) & ~15u;  // jtab: per chunk, first and last site of each 32-column half
    s.misc = s.bars + kNBars * 8;  // TMEM address, abort flag
    s.total = s.misc + 16;
    return s;
}

struct Blk {
    int i0, Bk;
};

__device__ __forceinline__ Blk blk_of(const PairArgs &p, long long kb)
{
    Blk g;
    g.i0 = (int)(kb % p.nb) * p.B;
    g.Bk = min(p.B, p.L - g.i0);
    return g;
}

__device__ __forceinline__ void blk_chunks(const PairArgs &p, long long kb, int &lo, int &hi)
{
    const Blk g = blk_of(p, kb);
    lo = g.i0 * p.q / kKC;
    hi = ((g.i0 + g.Bk) * p.q - 1) / kKC;
}

// One step of pair P's schedule in CTA r: n K chunks (n0 from c0, the rest
// from c1), main or delta, the own block t they feed, the block whose
// accumulator is complete after the step, the blocks a delta step carries,
// and what the generator waits for first (kind 1: the ready barrier of
// block wait_kb; kind 2: CTA 0's snapshot barrier after block wait_kb).
struct Seg {
    int n, n0, c0, c1, wait_kind;
    bool delta;
    long long t, wait_kb, commit_kb, d0, d1;
};

__device__ __forceinline__ int seg_chunk(const Seg &s, int k) { return k < s.n0 ? s.c0 + k : s.c1 + (k - s.n0); }

__device__ Seg seg_info(const PairArgs &p, long long P, int step, int r)
{
    Seg s;
    s.n = s.n0 = s.c0 = s.c1 = s.wait_kind = 0;
    s.delta = false;
    s.t = s.wait_kb = s.commit_kb = s.d0 = s.d1 = -1;
    const long long own = 2 * P + r;
    const bool has = own < p.nblocks;
    if (step == 0 || step == 2) {
        if (!has) return s;
        s.c0 = step == 0 ? 0 : p.X;
        s.n = s.n0 = step == 0 ? p.X : p.nK - p.X;
        s.t = own;
        if (step == 2 && P == 0 && r == 0) s.commit_kb = 0;
        return s;
    }
    if (P < 1) return s;
    s.delta = true;
    if (step == 1) {
        if (r != 1 || 2 * P - 1 >= p.nblocks) return s;
        int lo, hi;
        blk_chunks(p, 2 * P - 2, lo, hi);
        s.c0 = lo;
        s.n = s.n0 = hi - lo + 1;
        s.t = 2 * P - 1;
        s.d0 = 2 * P - 2;
        s.wait_kb = 2 * P - 2;
        s.wait_kind = 1;
        s.commit_kb = 2 * P - 1;
        return s;
    }
    if (!has) return s;
    int a0, a1, c0, c1;
    blk_chunks(p, 2 * P - 2, a0, a1);
    blk_chunks(p, 2 * P - 1, c0, c1);
    if (c0 <= a1 + 1 && a0 <= c1 + 1) {
        s.c0 = min(a0, c0);
        s.n = s.n0 = max(a1, c1) - s.c0 + 1;
    } else {  // the two blocks wrap around the end of a sweep
        s.c0 = a0;
        s.n0 = a1 - a0 + 1;
        s.c1 = c0;
        s.n = s.n0 + (c1 - c0 + 1);
    }
    s.t = own;
    s.d0 = 2 * P - 2;
    s.d1 = 2 * P - 1;
    s.wait_kb = 2 * P - 1;
    s.wait_kind = r == 0 ? 2 : 1;
    s.commit_kb = r == 0 ? own : -1;
    return s;
}

// Paired tensor cores (cta_group::2): one MMA stream serves both CTAs, so
// both run the same chunk sequence.  Step s of pair P has the chunks of the
// form above, in both CTAs: A and C the main chunks of pair P, B the delta
// chunks of block 2P-2, D those of blocks 2P-2 and 2P-1.  Per CTA r: the
// coupling rows it loads (block t; CTA 0's step B loads the rows of block
// 2P-2, whose accumulator is already drawn, and the MMA's CTA-0 half lands
// there harmlessly), the accumulator slot (jd & 1), what its generators wait
// for, and which CTAs' accumulators are complete after the step (bit r of
// commit_mask).  Blocks past the end (an odd block count) get the rows of a
// valid block and results nobody reads.
struct SegCg {
    Seg s;
    long long jd;
    int commit_mask;
};

__device__ SegCg seg_info_cg(const PairArgs &p, long long P, int step, int r)
{
    SegCg g;
    Seg &s = g.s;
    s.n = s.n0 = s.c0 = s.c1 = s.wait_kind = 0;
    s.delta = false;
    s.t = s.wait_kb = s.commit_kb = s.d0 = s.d1 = -1;
    g.jd = P;
    g.commit_mask = 0;
    if (step == 0 || step == 2) {
        if (2 * P >= p.nblocks) return g;
        s.c0 = step == 0 ? 0 : p.X;
        s.n = s.n0 = step == 0 ? p.X : p.nK - p.X;
        s.t = 2 * P + r;
        if (step == 2 && P == 0) g.commit_mask = 1;
        return g;
    }
    if (P < 1) return g;
    s.delta = true;
    if (step == 1) {
        if (2 * P - 1 >= p.nblocks) return g;
        int lo, hi;
        blk_chunks(p, 2 * P - 2, lo, hi);
        s.c0 = lo;
        s.n = s.n0 = hi - lo + 1;
        s.t = r == 1 ? 2 * P - 1 : 2 * P - 2;
        s.d0 = 2 * P - 2;
        s.wait_kb = 2 * P - 2;
        s.wait_kind = 1;
        g.jd = P - 1;
        g.commit_mask = 2;
        return g;
    }
    if (2 * P >= p.nblocks) return g;
    int a0, a1, c0, c1;
    blk_chunks(p, 2 * P - 2, a0, a1);
    blk_chunks(p, 2 * P - 1, c0, c1);
    if (c0 <= a1 + 1 && a0 <= c1 + 1) {
        s.c0 = min(a0, c0);
        s.n = s.n0 = max(a1, c1) - s.c0 + 1;
    } else {  // the two blocks wrap around the end of a sweep
        s.c0 = a0;
        s.n0 = a1 - a0 + 1;
        s.c1 = c0;
        s.n = s.n0 + (c1 - c0 + 1);
    }
    s.t = 2 * P + r;
    s.d0 = 2 * P - 2;
    s.d1 = 2 * P - 1;
    s.wait_kb = 2 * P - 1;
    s.wait_kind = r == 0 ? 2 : 1;
    g.commit_mask = 1;
    return g;
}

// tcgen05 forms for the paired tensor cores of a CTA pair.
__device__ __forceinline__ void mma_f16_cg2(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// Arrive (once) on the barrier at shared offset `bar` of every CTA in `mask`
// when all MMAs issued so far by this thread have completed.
__device__ __forceinline__ void mma_commit_mc(uint32_t bar, uint16_t mask)
{
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(bar),
        "h"(mask)
        : "memory");
}

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Categorical draw of the Gibbs conditional (Sec. 2.1) from beta*log2(e)-
// scaled fields H[0..q) (entries q..QC are -inf): weights 2^(H_a - max) by
// the hardware base-2 exponential (ex2.approx.ftz, a few ulp), prefix sums
// W_a, and the symbol is the number of prefix sums <= u * W_{q-1}, capped at
// q-1; since the prefix sums do not decrease this is the first a with
// u * W_{q-1} < W_a.  u = r24 / 2^24 from the chain's Philox counter.
template <int QC>
__device__ __forceinline__ int draw_symbol(float (&H)[QC], int q, uint32_t r24)
{
    static_assert(QC % 8 == 0 && QC <= 32, "QC: q rounded up to a multiple of 8");
    float m[8];  // maximum as a tree: QC -> 8 -> 4 -> 2 -> 1
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        m[a] = H[a];
#pragma unroll
        for (int k = 1; k < QC / 8; ++k) m[a] = fmaxf(m[a], H[a + 8 * k]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) m[a] = fmaxf(m[a], m[a + 4]);
    const float mx = fmaxf(fmaxf(m[0], m[2]), fmaxf(m[1], m[3]));
    float S = 0.0f;
#pragma unroll
    for (int a = 0; a < QC; ++a) {
        S += ex2_approx(H[a] - mx);
        H[a] = S;
    }
    const float thr = ((float)r24 * 5.9604644775390625e-8f) * S;
    int n = 0;
#pragma unroll
    for (int a = 0; a < QC; ++a) n += H[a] <= thr ? 1 : 0;
    return min(n, q - 1);
}

// The new symbol of a site: the Gibbs draw, or the Metropolis-Hastings step
// from the current symbol `cur` (w = bm_mh_word of the site).  H holds the
// fields scaled by beta*log2(e), entries past q masked.
template <int QC>
__device__ __forceinline__ int update_symbol(float (&H)[QC], int q, int cur, uint32_t w, int sampler)
{
    if (sampler != BM_SAMPLER_METROPOLIS) return draw_symbol<QC>(H, q, w);
    if (q < 2) return cur;
    int prop = (int)(w >> 24);
    prop += prop >= cur ? 1 : 0;
    float hp = 0.0f, hc = 0.0f;
#pragma unroll
    for (int a = 0; a < QC; ++a) {
        hp = a == prop ? H[a] : hp;
        hc = a == cur ? H[a] : hc;
    }
    return bm_mh_accept(hp, hc, w) ? prop : cur;
}

// BATCH: cluster k runs items[k] (its own model, tensor map and chain tile);
// otherwise every cluster runs the launch arguments on chains k*NC ...
// CG2: the two CTAs' tensor cores are paired (tcgen05 cta_group::2): CTA 0
// issues every MMA for both (M = 256: the coupling rows of block 2P in CTA 0
// and of block 2P+1 in CTA 1; N = NC chains, whose one-hot rows are split
// between the CTAs: CTA r generates and holds chains [r NC/2, (r+1) NC/2)).
// Each SM then generates and reads half of the one-hot operand per chunk.
// CTA 1's generators and drawers arrive on CTA 0's barriers; CTA 1's coupling
// tiles are reported to CTA 0 by a forwarding thread; CTA 0's commits
// multicast to both CTAs.
template <bool BATCH, int QC, bool CG2>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
    k_gibbs_pair(const __grid_constant__ CUtensorMap tm_one, const __grid_constant__ PairArgs p_one,
                 const PairItem *__restrict__ items)
{
    const PairItem *const item = BATCH ? items + (blockIdx.x >> 1) : nullptr;
    const PairArgs &p = BATCH ? item->a : p_one;
    const CUtensorMap *const tm_jp = BATCH ? &item->tm : &tm_one;
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = su32(smem_raw);
    unsigned char *base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    const int NCg = CG2 ? p.NC / 2 : p.NC;  // one-hot operand rows of this CTA
    const Smem lay = smem_layout(p.NC, p.Lp, p.B, p.nK, p.q, NCg);
    float *Hs = reinterpret_cast<float *>(base + lay.hs);
    uint8_t *st = base + lay.st;
    uint8_t *snap = base + lay.snap;
    const float4 *corr4 = reinterpret_cast<const float4 *>(base + lay.corr);
    float *hrow = reinterpret_cast<float *>(base + lay.hrow);
    unsigned short *jtab = reinterpret_cast<unsigned short *>(base + lay.jtab);
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + lay.bars);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(base + lay.misc);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(base + lay.misc + 4);
    const uint32_t full_a = su32(bars), empty_a = full_a + 8 * kNA;
    constexpr int NB = CG2 ? kNB2 : kNB;  // one-hot ring slots
    const uint32_t full_b = empty_a + 8 * kNA, empty_b = full_b + 8 * kNB2;
    const uint32_t acc_full = empty_b + 8 * kNB2;  // [2], own block j = kb/2 in slot j % 2
    const uint32_t acc_empty = acc_full + 16;     // [2]
    const uint32_t ready = acc_empty + 16;        // [2], states after block kb: barrier kb % 2
    const uint32_t snapready = ready + 16;        // CTA 0: next pair's snapshots taken
    const uint32_t corr_bar = snapready + 8;      // staged coupling blocks of the own block
    const uint32_t gen_done = corr_bar + 8;       // CTA 0: CTA 1's generators finished pair P's main chunks
    const uint32_t peer_full = gen_done + 8;      // CG2, CTA 0: [kNA] CTA 1's operands of the chunk in slot s
    const uint32_t fin = peer_full + 8 * kNA;     // CG2: every MMA of the launch completed
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r = (int)cluster_rank(), peer = r ^ 1;
    const int q = p.q, L = p.L, NC = p.NC, Lp = p.Lp;
    const int Sst = st_stride(Lp), Ssn = snap_stride(p.B);
    const size_t cta0 = BATCH ? (size_t)item->first : (size_t)(blockIdx.x >> 1) * NC;
    const long long nblocks = p.nblocks;
    const long long npairs = (nblocks + 1) / 2;
    auto snap_of = [&](long long kb) { return snap + (size_t)((((kb >> 1) & 1) * 2 + (kb & 1)) * NC) * Ssn; };

    if (tid == 0) {
        for (int s = 0; s < kNA; ++s) {
            mbar_init(full_a + 8 * s, 1);
            mbar_init(empty_a + 8 * s, 1);
        }
        for (int s = 0; s < NB; ++s) {
            mbar_init(full_b + 8 * s, kGenWarps);
            mbar_init(empty_b + 8 * s, 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(acc_full + 8 * s, 1);
            mbar_init(acc_empty + 8 * s, CG2 ? 2 * kDrawWarps : kDrawWarps);
            mbar_init(ready + 8 * s, kDraw);
        }
        mbar_init(snapready, kDraw);
        mbar_init(corr_bar, 1);
        mbar_init(gen_done, kGenWarps);
        for (int s = 0; s < kNA; ++s) mbar_init(peer_full + 8 * s, 1);
        mbar_init(fin, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        if (CG2) {  // one warp of each CTA of the pair; both get the same columns
            asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                         "r"(p.tmem_cols)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
        } else {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                         "r"(p.tmem_cols)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
    }
    for (int k = tid; k < NC * Lp; k += kThreads) {
        const int c = k / Lp, x = k - c * Lp;
        const size_t m = cta0 + c;
        st[c * Sst + x] = (m < (size_t)p.M && x < L) ? p.states[m * L + x] : 0;
    }
    for (int c = tid; c < p.nK; c += kThreads) {
        const int k0 = c * kKC;
        jtab[4 * c] = (unsigned short)min(L - 1, k0 / q);
        jtab[4 * c + 1] = (unsigned short)min(L - 1, (k0 + kKC / 2 - 1) / q);
        jtab[4 * c + 2] = (unsigned short)min(L - 1, (k0 + kKC / 2) / q);
        jtab[4 * c + 3] = (unsigned short)min(L - 1, (k0 + kKC - 1) / q);
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
    cluster_sync_all();  // both CTAs' barriers are initialised before any remote arrival
    const uint32_t tmem = *tmem_slot;

    // Stage the in-block coupling blocks of block kb (its pairs pi > pj are
    // the first Bk(Bk-1)/2 slots of its Jc entry): one bulk copy.
    auto stage_corr = [&](long long kb) {
        const Blk g = blk_of(p, kb);
        const uint32_t row = (uint32_t)q * (uint32_t)q4_of(q);
        const uint32_t bytes = (uint32_t)corr_slots(g.Bk) * row * 4u;
        mbar_expect_tx(corr_bar, bytes);
        if (bytes > 0)
            bulk_g2s(su32(base + lay.corr), p.Jc + (size_t)(kb % p.nb) * corr_slots(p.B) * row, bytes, corr_bar);
    };

    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            long long issued = 0;
            int sa = 0, lap = 0;
            bool ok = true;
            for (long long P = 0; P <= npairs && ok; ++P)
                for (int step = 0; step < 4 && ok; ++step) {
                    const Seg sg = CG2 ? seg_info_cg(p, P, step, r).s : seg_info(p, P, step, r);
                    const int r0 = sg.n > 0 ? (int)(sg.t % p.nb) * kRowsA : 0;
                    for (int k = 0; k < sg.n && ok; ++k) {
                        const int c = seg_chunk(sg, k);
                        if (lap > 0 && !mbar_wait(empty_a + 8 * sa, (uint32_t)((lap - 1) & 1), abort_flag, p.err)) {
                            ok = false;
                            break;
                        }
                        const uint32_t dst = su32(base + lay.a + sa * kSlotA), bar = full_a + 8 * sa;
                        if (CG2) {  // both CTAs' tiles count on CTA 0's barrier of the slot
                            if (r == 0) mbar_expect_tx(bar, 2u * (uint32_t)kSlotA);
                            tma_load_3d_cg2(dst, tm_jp, 0, r0, 2 * c, peer_addr(bar, 0));
                        } else {
                            mbar_expect_tx(bar, (uint32_t)kSlotA);
                            tma_load_3d(dst, tm_jp, 0, r0, 2 * c, bar);  // hi slab then lo slab of 128 rows
                        }
                        ++issued;
                        if (++sa == kNA) {
                            sa = 0;
                            ++lap;
                        }
                    }
                }
            if (*abort_flag) {  // let the copies in flight land before exit
                if (!CG2 || r == 0) {
                    volatile int no_abort = 0;
                    for (long long u = issued > kNA ? issued - kNA : 0; u < issued; ++u)
                        mbar_wait(full_a + 8 * (int)(u % kNA), (uint32_t)((u / kNA) & 1), &no_abort, p.err);
                } else {
                    __nanosleep(100000);  // this CTA's tiles are counted on CTA 0's barriers
                }
            }
        }
    } else if (warp == 1 && CG2) {
        // ------------------------------------------------------------ paired MMA issuer (CTA 0)
        if (lane == 0 && r == 0) {
            // kind::f16: D F32 (bit 4), A = B = F16, K-major, N >> 3 at 17, M >> 4 at 24; M = 256
            // across the pair (128 coupling rows per CTA), N = NC (NC/2 one-hot rows per CTA).
            const uint32_t idesc = (1u << 4) | ((uint32_t)(NC >> 3) << 17) | ((uint32_t)((2 * kRowsA) >> 4) << 24);
            int sa = 0, sb = 0;
            uint32_t pha = 0, phb = 0;
            bool ok = true;
            for (long long P = 0; P <= npairs && ok; ++P)
                for (int step = 0; step < 4 && ok; ++step) {
                    const SegCg gc = seg_info_cg(p, P, step, 0);
                    const Seg &sg = gc.s;
                    const long long j = gc.jd;
                    for (int k = 0; k < sg.n && ok; ++k) {
                        const int c = seg_chunk(sg, k);
                        const bool first = !sg.delta && c == 0;
                        if (!mbar_wait(full_b + 8 * sb, phb, abort_flag, p.err) ||
                            !mbar_wait(full_a + 8 * sa, pha, abort_flag, p.err)) {
                            ok = false;
                            break;
                        }
                        // CTA 1's one-hot rows of this chunk (relayed by its forwarding
                        // thread; slot sa of the coupling ring, same phase); its coupling
                        // tile is counted on full_a above
                        if (!mbar_wait_cl(peer_full + 8 * sa, pha, abort_flag, p.err)) {
                            ok = false;
                            break;
                        }
                        if (first && j >= 2 &&
                            !mbar_wait_cl(acc_empty + 8 * (int)(j & 1), (uint32_t)(((j - 2) >> 1) & 1), abort_flag,
                                          p.err)) {
                            ok = false;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t bb = su32(base + lay.b + sb * NCg * 128);
                        const uint32_t ah = su32(base + lay.a + sa * kSlotA), al = ah + kTileA;
                        const uint32_t dcol = tmem + (uint32_t)(j & 1) * p.acc_stride;
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint64_t bd = desc_noswz(bb + kk * 256);
                            mma_f16_cg2(dcol, desc_sw128(ah + kk * 32), bd, idesc, (first && kk == 0) ? 0u : 1u);
                            mma_f16_cg2(dcol, desc_sw128(al + kk * 32), bd, idesc, 1u);
                        }
                        // one commit per chunk frees both its coupling slot and its one-hot
                        // slot (the generators wait on the coupling ring's barriers)
                        mma_commit_mc(empty_a + 8 * sa, 3);
                        if (++sa == kNA) {
                            sa = 0;
                            pha ^= 1u;
                        }
                        if (++sb == NB) {
                            sb = 0;
                            phb ^= 1u;
                        }
                    }
                    if (ok && gc.commit_mask) mma_commit_mc(acc_full + 8 * (int)(j & 1), (uint16_t)gc.commit_mask);
                }
            mma_commit_mc(fin, 3);  // teardown waits for every MMA of the launch, in both CTAs
        } else if (lane == 0) {
            // CTA 1: relay, chunk by chunk, that this CTA's one-hot rows are in
            // place (one arrival on CTA 0's barrier of the chunk's coupling
            // slot; its coupling tiles count on CTA 0's full_a directly).  A slot's barrier cannot move on by two
            // phases before CTA 0 has consumed the chunk: the chunk kNA later
            // needs this slot refilled, which waits for that chunk's MMAs.
            const uint32_t pf0 = peer_addr(peer_full, 0);
            long long total = 0;
            for (long long P = 0; P <= npairs; ++P)
                for (int step = 0; step < 4; ++step) total += seg_info_cg(p, P, step, 1).s.n;
            for (long long k = 0; k < total; ++k) {
                if (!mbar_wait(full_b + 8 * (int)(k % NB), (uint32_t)((k / NB) & 1), abort_flag, p.err)) break;
                mbar_arrive_peer_relaxed(pf0 + 8 * (uint32_t)(k % kNA));
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            // kind::f16: D F32 (bit 4), A = B = F16, K-major, N >> 3 at 17, M >> 4 at 24.
            const uint32_t idesc = (1u << 4) | ((uint32_t)(NC >> 3) << 17) | ((uint32_t)(kRowsA >> 4) << 24);
            int sa = 0, sb = 0;
            uint32_t pha = 0, phb = 0;
            bool ok = true;
            for (long long P = 0; P <= npairs && ok; ++P)
                for (int step = 0; step < 4 && ok; ++step) {
                    const Seg sg = seg_info(p, P, step, r);
                    const long long j = sg.t >> 1;  // own block index
                    for (int k = 0; k < sg.n && ok; ++k) {
                        const int c = seg_chunk(sg, k);
                        const bool first = !sg.delta && c == 0;
                        if (!mbar_wait(full_b + 8 * sb, phb, abort_flag, p.err)) {
                            ok = false;
                            break;
                        }
                        if (!mbar_wait(full_a + 8 * sa, pha, abort_flag, p.err)) {
                            ok = false;
                            break;
                        }
                        if (first && j >= 2 &&
                            !mbar_wait(acc_empty + 8 * (int)(j & 1), (uint32_t)(((j - 2) >> 1) & 1), abort_flag,
                                       p.err)) {
                            ok = false;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t bb = su32(base + lay.b + sb * NC * 128);
                        const uint32_t ah = su32(base + lay.a + sa * kSlotA), al = ah + kTileA;
                        const uint32_t dcol = tmem + (uint32_t)(j & 1) * p.acc_stride;
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint64_t bd = desc_noswz(bb + kk * 256);
                            mma_f16(dcol, desc_sw128(ah + kk * 32), bd, idesc, (first && kk == 0) ? 0u : 1u);
                            mma_f16(dcol, desc_sw128(al + kk * 32), bd, idesc, 1u);
                        }
                        mma_commit(empty_a + 8 * sa);  // frees the chunk's coupling and one-hot slots
                        if (++sa == kNA) {
                            sa = 0;
                            pha ^= 1u;
                        }
                        if (++sb == NB) {
                            sb = 0;
                            phb ^= 1u;
                        }
                    }
                    if (ok && sg.commit_kb >= 0) mma_commit(acc_full + 8 * (int)((sg.commit_kb >> 1) & 1));
                }
        }
    } else if (warp < 2 + kDrawWarps) {
        // ------------------------------------------------------------ drawers (warps 2-6)
        // Uniform control flow: every drawer runs the whole loop nest and meets
        // every named barrier; after an abort the work is skipped.
        const int w = tid - 64;                 // 0..kDraw-1, chain w
        const bool tm_reader = warp < 6;        // warps 2-5 cover TMEM lane quarters 2, 3, 0, 1
        const int lane_base = 32 * (warp & 3);
        const int row = lane_base + lane;
        const int HS = hs_stride(q), qv = q4_of(q) >> 2;  // float4s per padded row
        const uint32_t st_peer = peer_addr(su32(st), (uint32_t)peer);
        const uint32_t ready_peer = peer_addr(ready, (uint32_t)peer);
        bool ok = true;
        long long staged = 0;
        if (w == 0 && r < nblocks) {
            stage_corr(r);
            staged = 1;
        }
        for (long long kb = r; kb < nblocks; kb += 2) {
            const long long j = kb >> 1;
            const Blk g = blk_of(p, kb);
            const int slot = (int)(j & 1);
            const uint64_t sweep = p.sweep0 + (uint64_t)(kb / p.nb);
            // the block's Philox numerators (independent of the states) while the
            // accumulator fills, two independent streams at a time
            uint32_t ur[kBmax];
            if (w < NC) {
                const uint64_t m = p.chain0 + cta0 + w;
                for (int pp = 0; pp < g.Bk; pp += 2) {
                    const uint64_t i0 = (uint64_t)(g.i0 + pp);
                    const uint32_t u0 = p.sampler == BM_SAMPLER_METROPOLIS ? bm_mh_word(p.seed, m, sweep, i0, q)
                                                                          : bm_u24(p.seed, m, sweep, i0, 0);
                    const uint32_t u1 = p.sampler == BM_SAMPLER_METROPOLIS ? bm_mh_word(p.seed, m, sweep, i0 + 1, q)
                                                                          : bm_u24(p.seed, m, sweep, i0 + 1, 0);
                    ur[pp] = u0;
                    if (pp + 1 < g.Bk) ur[pp + 1] = u1;
                }
            }
            if (ok && !mbar_wait(acc_full + 8 * slot, (uint32_t)((j >> 1) & 1), abort_flag, p.err)) ok = false;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int k = w; k < g.Bk * q; k += kDraw) hrow[k] = p.h[(size_t)g.i0 * q + k];
            if (ok && !mbar_wait(corr_bar, (uint32_t)(j & 1), abort_flag, p.err)) ok = false;
            ok = !named_bar_or(1, kDraw, !ok || *abort_flag);
            const uint8_t *old = snap_of(kb);
            const uint32_t tacc = tmem + ((uint32_t)lane_base << 16) + (uint32_t)slot * p.acc_stride;
            for (int pp = 0; pp < g.Bk && ok; ++pp) {
                const int r0 = pp * q;
                if (tm_reader && lane_base < r0 + q && lane_base + 32 > r0) {
                    const bool mine = row >= r0 && row < r0 + q;
                    const float hv = mine ? hrow[row] : 0.0f;
                    // up to 48 columns (chains) in flight per wait: 16-column loads
                    // issued back to back, then one wait (NC is a multiple of 16)
                    for (int c0 = 0; c0 < NC; c0 += 48) {
                        const int nc = min(48, NC - c0);
                        uint32_t v[3][16];
#pragma unroll
                        for (int u = 0; u < 3; ++u)
                            if (16 * u < nc) tmem_ld16(tacc + (uint32_t)(c0 + 16 * u), v[u]);
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                        if (mine) {
#pragma unroll
                            for (int u = 0; u < 3; ++u)
                                if (16 * u < nc) {
#pragma unroll
                                    for (int e = 0; e < 16; ++e)
                                        Hs[(c0 + 16 * u + e) * HS + (row - r0)] = hv + __uint_as_float(v[u][e]);
                                }
                        }
                    }
                }
                named_bar_sync(1, kDraw);
                const int i = g.i0 + pp;
                if (w < NC) {
                    const int ch = w;
                    const uint32_t r24 = ur[pp];
                    // QC/4 float4s per row: past q the entries are masked below
                    float H[QC];
                    const float4 *hs4 = reinterpret_cast<const float4 *>(Hs + ch * HS);
#pragma unroll
                    for (int a4 = 0; a4 < QC / 4; ++a4) {
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
                        for (int a4 = 0; a4 < QC / 4; ++a4) {  // past q4: the next row or the h rows, masked
                            const float4 vn = rn[a4], vo = ro[a4];
                            H[4 * a4] += vn.x - vo.x;
                            H[4 * a4 + 1] += vn.y - vo.y;
                            H[4 * a4 + 2] += vn.z - vo.z;
                            H[4 * a4 + 3] += vn.w - vo.w;
                        }
                    }
#pragma unroll
                    for (int a = 0; a < QC; ++a) H[a] = a < q ? H[a] * p.beta_l2e : -INFINITY;
                    st[ch * Sst + i] = (uint8_t)update_symbol<QC>(H, q, st[ch * Sst + i], r24, p.sampler);
                }
                named_bar_sync(1, kDraw);  // Hs is rewritten for the next site
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) {
                if (CG2 && r == 1)
                    mbar_arrive_peer(peer_addr(acc_empty + 8 * (uint32_t)slot, 0));
                else
                    mbar_arrive(acc_empty + 8 * slot);
            }
            named_bar_sync(1, kDraw);  // the staged coupling blocks are free again
            if (w == 0 && ok && !*abort_flag && kb + 2 < nblocks) {
                stage_corr(kb + 2);
                ++staged;
            }
            // CTA 1: the next pair's snapshots, before block kb is published
            // (CTA 0 starts rewriting block kb+1's sites once it has it).
            if (r == 1 && kb + 1 < nblocks) {
                if (ok && !mbar_wait_cl(ready + 8 * (int)((kb - 1) & 1), (uint32_t)(((kb - 1) >> 1) & 1), abort_flag,
                                        p.err))
                    ok = false;
                if (ok && w < NC)
                    for (long long nb2 = kb + 1; nb2 <= kb + 2 && nb2 < nblocks; ++nb2) {
                        const Blk gn = blk_of(p, nb2);
                        uint8_t *sn = snap_of(nb2) + w * Ssn;
                        for (int x = 0; x < gn.Bk; ++x) sn[x] = st[w * Sst + gn.i0 + x];
                    }
            }
            // Copy block kb's new states into the peer's copy.  CTA 0 first waits
            // until CTA 1's generators have finished pair j's main chunks, which
            // still read block kb's pre-redraw states from CTA 1's copy.
            if (r == 0 && ok && !mbar_wait_cl(gen_done, (uint32_t)(j & 1), abort_flag, p.err)) ok = false;
            if (ok && w < NC)
                for (int x = 0; x < g.Bk; ++x)
                    st_cluster_u8(st_peer + (uint32_t)(w * Sst + g.i0 + x), (unsigned short)st[w * Sst + g.i0 + x]);
            // publish block kb: own generator and the peer
            mbar_arrive(ready + 8 * (int)(kb & 1));
            mbar_arrive_peer(ready_peer + 8 * (uint32_t)(kb & 1));
            // CTA 0: the next pair's snapshots once block kb+1 has arrived
            if (r == 0 && kb + 1 < nblocks) {
                if (ok && !mbar_wait_cl(ready + 8 * (int)((kb + 1) & 1), (uint32_t)(((kb + 1) >> 1) & 1), abort_flag,
                                        p.err))
                    ok = false;
                if (ok && w < NC)
                    for (long long nb2 = kb + 2; nb2 <= kb + 3 && nb2 < nblocks; ++nb2) {
                        const Blk gn = blk_of(p, nb2);
                        uint8_t *sn = snap_of(nb2) + w * Ssn;
                        for (int x = 0; x < gn.Bk; ++x) sn[x] = st[w * Sst + gn.i0 + x];
                    }
                mbar_arrive(snapready);
            }
        }
        if (!ok) *abort_flag = 1;
        if (w == 0 && *abort_flag && staged > 0) {
            volatile int no_abort = 0;
            mbar_wait(corr_bar, (uint32_t)((staged - 1) & 1), &no_abort, p.err);
        }
    } else {
        // ------------------------------------------------------------ generators (warps 7-11)
        // One thread per operand row; with paired tensor cores (NC/2 rows per
        // CTA) two threads per row, each writing one 32-column half of a chunk.
        // kNS bounds the sites a thread's columns touch for alphabets of this
        // QC (q > QC - 8): chunks within it take the unrolled path.
        constexpr int kNS = QC == 8 ? 8 : (CG2 ? 32 : 64) / (QC - 7) + 2 > 8 ? 8 : (CG2 ? 32 : 64) / (QC - 7) + 2;
        const int gt = tid - 64 - kDraw;             // 0..kGen-1
        const int w = CG2 ? gt >> 1 : gt;            // operand row of this CTA
        const int cb = CG2 ? 32 * (gt & 1) : 0;      // chunk columns [cb, ce) of this thread
        const int ce = CG2 ? cb + 32 : kKC;
        const bool own = w < NCg;
        const int ch = (CG2 ? r * NCg : 0) + (own ? w : 0);  // its chain
        unsigned char *const row0 = base + lay.b + noswz_off(own ? w : 0, 0);
        const uint8_t *const strow = st + ch * Sst;
        const int wrow = ch * Ssn;
        const uint32_t gen_done_peer = peer_addr(gen_done, (uint32_t)peer);
        int sb = 0, lap = 0;
        long long gk = 0;  // chunks generated so far
        bool ok = true;
        for (long long P = 0; P <= npairs && ok; ++P) {
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
                const Seg sg = CG2 ? seg_info_cg(p, P, step, r).s : seg_info(p, P, step, r);
                if (sg.n > 0 && sg.wait_kind != 0) {
                    const uint32_t bar = sg.wait_kind == 1 ? ready + 8 * (uint32_t)(sg.wait_kb & 1) : snapready;
                    if (!mbar_wait_cl(bar, (uint32_t)((sg.wait_kb >> 1) & 1), abort_flag, p.err)) {
                        ok = false;
                        break;
                    }
                }
                // Main chunks touching at most 8 sites (q >= 8): the state bytes of
                // the row's nonzeros are loaded one chunk ahead (before the previous
                // chunk's slot wait and stores), so their latency is hidden and only
                // the stores remain after the wait.
                auto chunk_sites = [&](int kk, int &jlo, int &jhi, bool &fast) {
                    const int c = seg_chunk(sg, kk);
                    jlo = jtab[4 * c + (CG2 ? 2 * (cb >> 5) : 0)];
                    jhi = jtab[4 * c + (CG2 ? 2 * (cb >> 5) + 1 : 3)];
                    fast = !sg.delta && jhi - jlo < kNS;
                };
                auto load_states = [&](int jlo, int jhi, bool fast, int (&sv)[kNS]) {
#pragma unroll
                    for (int t = 0; t < kNS; ++t) {
                        const int jj = jlo + t;
                        sv[t] = -1;
                        if (fast && own && jj <= jhi) {
                            const uint8_t *src = strow + jj;
                            src = (jj >= s0lo && jj < s0hi) ? ps0 + (jj - s0lo) : src;
                            src = (jj >= s1lo && jj < s1hi) ? ps1 + (jj - s1lo) : src;
                            sv[t] = *src;
                        }
                    }
                };
                int nxt_lo = 0, nxt_hi = 0, nxt_sv[kNS];
                bool nxt_fast = false;
                if (sg.n > 0) {
                    chunk_sites(0, nxt_lo, nxt_hi, nxt_fast);
                    load_states(nxt_lo, nxt_hi, nxt_fast, nxt_sv);
                }
                for (int k = 0; k < sg.n; ++k) {
                    const int c = seg_chunk(sg, k);
                    const int k0 = c * kKC;
                    const int jlo = nxt_lo, jhi = nxt_hi;
                    const bool fast = nxt_fast;
                    int fpos[kNS];
#pragma unroll
                    for (int t = 0; t < kNS; ++t) fpos[t] = nxt_sv[t] >= 0 ? (jlo + t) * q + nxt_sv[t] - k0 : -1;
                    if (k + 1 < sg.n) {
                        chunk_sites(k + 1, nxt_lo, nxt_hi, nxt_fast);
                        load_states(nxt_lo, nxt_hi, nxt_fast, nxt_sv);
                    }
                    // one-hot slot sb is free once the MMAs of chunk gk - NB completed:
                    // the commit of that chunk on the coupling ring's barrier.  NB <= kNA,
                    // so that barrier cannot have moved on by a further phase (that
                    // chunk's successor there needs a one-hot tile not yet written).
                    if (gk >= NB && !mbar_wait(empty_a + 8 * (int)((gk - NB) % kNA),
                                               (uint32_t)(((gk - NB) / kNA) & 1), abort_flag, p.err)) {
                        ok = false;
                        break;
                    }
                    ++gk;
                    unsigned char *rowp = row0 + sb * NCg * 128;
                    if (own) {
#pragma unroll
                        for (int pc = 0; pc < 8; ++pc)
                            if (pc * 8 >= cb && pc * 8 < ce)
                                *reinterpret_cast<uint4 *>(rowp + pc * 128) = make_uint4(0, 0, 0, 0);
                        if (fast) {
#pragma unroll
                            for (int t = 0; t < kNS; ++t) {
                                const int pos = fpos[t];
                                if (pos >= cb && pos < ce)
                                    *reinterpret_cast<unsigned short *>(rowp + (pos >> 3) * 128 + (pos & 7) * 2) =
                                        0x3c00u;
                            }
                        } else if (!sg.delta) {
                            for (int jj = jlo; jj <= jhi; ++jj) {
                                const int sj = (jj >= s0lo && jj < s0hi)   ? ps0[jj - s0lo]
                                               : (jj >= s1lo && jj < s1hi) ? ps1[jj - s1lo]
                                                                           : strow[jj];
                                const int pos = jj * q + sj - k0;
                                if (pos >= cb && pos < ce)
                                    *reinterpret_cast<unsigned short *>(rowp + (pos >> 3) * 128 + (pos & 7) * 2) =
                                        0x3c00u;
                            }
                        } else {
                            for (int u = 0; u < 2; ++u) {
                                const long long db = u == 0 ? sg.d0 : sg.d1;
                                if (db < 0) continue;
                                const Blk gd = blk_of(p, db);
                                const uint8_t *po = (u == 0 ? ps0 : ps1);  // d0 = 2P-2, d1 = 2P-1
                                // only the block's sites inside this thread's columns
                                const int x0 = max(0, jlo - gd.i0), x1 = min(gd.Bk, jhi - gd.i0 + 1);
                                for (int x = x0; x < x1; ++x) {
                                    const int jj = gd.i0 + x;
                                    const int sn = strow[jj], so = po[x];
                                    if (sn == so) continue;
                                    const int pn = jj * q + sn - k0, pd = jj * q + so - k0;
                                    if (pn >= cb && pn < ce)
                                        *reinterpret_cast<unsigned short *>(rowp + (pn >> 3) * 128 + (pn & 7) * 2) =
                                            0x3c00u;
                                    if (pd >= cb && pd < ce)
                                        *reinterpret_cast<unsigned short *>(rowp + (pd >> 3) * 128 + (pd & 7) * 2) =
                                            0xbc00u;
                                }
                            }
                        }
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(full_b + 8 * sb);
                    if (++sb == NB) {
                        sb = 0;
                        ++lap;
                    }
                }
                // CTA 1: pair P's main chunks are read; CTA 0 may now overwrite
                // block 2P's sites in this CTA's copy of the states
                if (ok && r == 1 && step == 2 && 2 * P < nblocks) {
                    __syncwarp();
                    if (lane == 0) mbar_arrive_peer(gen_done_peer);
                }
            }
        }
        if (!ok) *abort_flag = 1;
    }
    if (CG2 && warp == 1 && lane == 0) {  // CTA 0's MMAs write both CTAs' tensor memory
        volatile int no_abort = 0;
        mbar_wait(fin, 0, &no_abort, p.err);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (CG2) {
        cluster_sync_all();
        if (warp == 1)
            asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.tmem_cols)
                         : "memory");
    } else if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.tmem_cols)
                     : "memory");
    }
    // No remote store or arrival into either CTA is in flight past this
    // barrier; then each CTA reads the other's abort flag, and the second
    // barrier keeps both CTAs resident until those reads are done.
    cluster_sync_all();
    const bool bad = *abort_flag != 0 || ld_cluster_u32(peer_addr(su32((const void *)abort_flag), (uint32_t)peer)) != 0;
    cluster_sync_all();
    if (bad) return;
    const int half = NC / 2;  // CTA r writes back chains 2c + r
    for (int k = tid; k < half * L; k += kThreads) {
        const int cc = k / L, x = k - cc * L;
        const int c = 2 * cc + r;
        const size_t m = cta0 + c;
        if (m < (size_t)p.M) p.states[m * L + x] = st[c * Sst + x];
    }
}

// ---------------------------------------------------------------------------
// Tensor-memory operand form.  Same schedule, exchange and snapshots as
// k_gibbs_pair, with the roles of the MMA operands swapped: the one-hot
// states are the A operand (M = 128 chains, one TMEM lane per chain), written
// by the generators into tensor memory with tcgen05.st, and the coupling
// tile is the B operand (N = the block's rows (i,a) rounded up to 16, K-major
// 128B-swizzled in shared memory as loaded by TMA).  The accumulator then
// holds one chain per TMEM lane and one row (i,a) per column, so each drawer
// thread reads its own chain's fields of a site straight from TMEM.  Per
// 64-column K chunk the shared-memory traffic is the 32 KB coupling tile
// written by TMA and read once by the MMAs; the one-hot operand never touches
// shared memory.
//
// TMEM (512 columns): accumulators of own blocks j = kb/2 in columns
// [128 (j%2), +128); one-hot ring slot s in columns [256 + 32 s, +32), two
// fp16 K elements per column (the lower half holds the even element).
// Warps: 0 TMA producer; 1 TMEM allocation and the MMA thread; 2-5 drawers
// (chain 32 (warp%4) + lane, the TMEM lane quarter a warp may access); 6-9
// generators (same chain mapping).
// ---------------------------------------------------------------------------
constexpr int kTmNC = 128;  // chains per cluster = MMA M
constexpr int kTmNAmax = 4;
constexpr int kTmNB = 4;
constexpr int kTmDraw = 128, kTmGen = 128;
constexpr int kTmThreads = 64 + kTmDraw + kTmGen;
constexpr uint32_t kTmCols = 512, kTmAccCols = 128, kTmOneHotCol = 256;
constexpr int kTmNBars = 2 * kTmNAmax + 2 * kTmNB + 2 + 2 + 2 + 1 + 1 + 1;
constexpr int kTmUrS = kBmax + 1;  // row stride (words) of the per-chain uniform table

__host__ __device__ inline Smem smem_layout_tm(int na, int Lp, int B, int nK, int q)
{
    Smem s;
    s.a = 0;
    s.b = s.a + na * kSlotA;  // no shared-memory one-hot ring or field rows
    s.st = s.b;
    s.snap = s.st + kTmNC * st_stride(Lp);
    s.corr = (s.snap + 4 * kTmNC * snap_stride(B) + 15) & ~15u;
    s.hrow = s.corr + (uint32_t)corr_slots(B) * q * q4_of(q) * 4;  // [2][128]: h rows of own blocks j % 2
    s.hs = s.hrow + 2 * kRowsA * 4;                                  // uniforms: [chain][kTmUrS]
    s.jtab = s.hs + kTmNC * kTmUrS * 4;
    s.bars = (s.jtab + nK * 4 + 15) & ~15u;
    s.misc = s.bars + kTmNBars * 8;
    s.total = s.misc + 16;
    return s;
}

__device__ __forceinline__ void mma_f16_ts(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ uint32_t tmem_ld1(uint32_t taddr)
{
    uint32_t v;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(v) : "r"(taddr));
    return v;
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]),
        "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]),
        "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]),
        "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
        : "memory");
}

// The 32 registers (fp16 pairs, even element in the lower half) of a 64-element
// one-hot row from bit masks of its +1 (0x3c00) and -1 (0xbc00) entries.  Per
// 4-element nibble x: x * 0x00204081 = x + (x << 7) + (x << 14) + (x << 21)
// holds four disjoint copies of x, in which bit b of copy b sits at bit 8b;
// & 0x01010101 keeps those, so byte b is bit b of x.  The bytes are scaled to
// the fp16 high bytes 0x3c / 0xbc and moved into place by byte permutes.
template <bool MINUS>
__device__ __forceinline__ void onehot_regs(uint64_t plus, uint64_t minus, uint32_t (&v)[32])
{
#pragma unroll
    for (int n = 0; n < 16; ++n) {
        const uint32_t xp = (uint32_t)(plus >> (4 * n)) & 0xfu;
        uint32_t w = ((xp * 0x00204081u) & 0x01010101u) * 0x3cu;
        if (MINUS) {
            const uint32_t xm = (uint32_t)(minus >> (4 * n)) & 0xfu;
            w += ((xm * 0x00204081u) & 0x01010101u) * 0xbcu;
        }
        v[2 * n] = __byte_perm(w, 0u, 0x1404);      // bytes: 0, w0, 0, w1
        v[2 * n + 1] = __byte_perm(w, 0u, 0x3424);  // bytes: 0, w2, 0, w3
    }
}

// 1 << n, and 0 when n (as an unsigned amount) is 32 or more: PTX clamps
// the shift amount, so out-of-range positions need no test.
__device__ __forceinline__ uint32_t bit_at(int n)
{
    uint32_t r;
    asm("shl.b32 %0, 1, %1;" : "=r"(r) : "r"(n));
    return r;
}

template <bool BATCH, int QC>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kTmThreads, 1)
    k_gibbs_pair_tm(const __grid_constant__ CUtensorMap tm_one, const __grid_constant__ PairArgs p_one,
                    const PairItem *__restrict__ items)
{
    const PairItem *const item = BATCH ? items + (blockIdx.x >> 1) : nullptr;
    const PairArgs &p = BATCH ? item->a : p_one;
    const CUtensorMap *const tm_jp = BATCH ? &item->tm : &tm_one;
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = su32(smem_raw);
    unsigned char *base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    const int na = p.na;
    const Smem lay = smem_layout_tm(na, p.Lp, p.B, p.nK, p.q);
    uint8_t *st = base + lay.st;
    uint8_t *snap = base + lay.snap;
    const float4 *corr4 = reinterpret_cast<const float4 *>(base + lay.corr);
    float *hrow = reinterpret_cast<float *>(base + lay.hrow);
    unsigned short *jtab = reinterpret_cast<unsigned short *>(base + lay.jtab);
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + lay.bars);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(base + lay.misc);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(base + lay.misc + 4);
    const uint32_t full_a = su32(bars), empty_a = full_a + 8 * kTmNAmax;
    const uint32_t full_b = empty_a + 8 * kTmNAmax, empty_b = full_b + 8 * kTmNB;
    const uint32_t acc_full = empty_b + 8 * kTmNB;  // [2], own block j = kb/2 in slot j % 2
    const uint32_t acc_empty = acc_full + 16;       // [2]
    const uint32_t ready = acc_empty + 16;          // [2], states after block kb: barrier kb % 2
    const uint32_t snapready = ready + 16;          // CTA 0: next pair's snapshots taken
    const uint32_t corr_bar = snapready + 8;        // staged coupling blocks of the own block
    const uint32_t gen_done = corr_bar + 8;         // CTA 0: CTA 1's generators finished pair P's main chunks
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r = (int)cluster_rank(), peer = r ^ 1;
    const int q = p.q, L = p.L, Lp = p.Lp;
    constexpr int NC = kTmNC;
    const int Sst = st_stride(Lp), Ssn = snap_stride(p.B);
    const size_t cta0 = BATCH ? (size_t)item->first : (size_t)(blockIdx.x >> 1) * NC;
    const long long nblocks = p.nblocks;
    const long long npairs = (nblocks + 1) / 2;
    auto snap_of = [&](long long kb) { return snap + (size_t)((((kb >> 1) & 1) * 2 + (kb & 1)) * NC) * Ssn; };

    if (tid == 0) {
        for (int s = 0; s < kTmNAmax; ++s) {
            mbar_init(full_a + 8 * s, 1);
            mbar_init(empty_a + 8 * s, 1);
        }
        for (int s = 0; s < kTmNB; ++s) {
            mbar_init(full_b + 8 * s, kTmGen / 32);
            mbar_init(empty_b + 8 * s, 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(acc_full + 8 * s, 1);
            mbar_init(acc_empty + 8 * s, kTmDraw / 32);
            mbar_init(ready + 8 * s, kTmDraw);
        }
        mbar_init(snapready, kTmDraw);
        mbar_init(corr_bar, 1);
        mbar_init(gen_done, kTmGen / 32);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(kTmCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int k = tid; k < NC * Lp; k += kTmThreads) {
        const int c = k / Lp, x = k - c * Lp;
        const size_t m = cta0 + c;
        st[c * Sst + x] = (m < (size_t)p.M && x < L) ? p.states[m * L + x] : 0;
    }
    for (int c = tid; c < p.nK; c += kTmThreads) {
        const int k0 = c * kKC;
        jtab[2 * c] = (unsigned short)min(L - 1, k0 / q);
        jtab[2 * c + 1] = (unsigned short)min(L - 1, (k0 + kKC - 1) / q);
    }
    __syncthreads();
    for (long long kb = 0; kb < 2 && kb < nblocks; ++kb) {  // snapshots of pair 0
        const Blk g = blk_of(p, kb);
        uint8_t *sn = snap_of(kb);
        for (int k = tid; k < NC * g.Bk; k += kTmThreads) {
            const int c = k / g.Bk, x = k - c * g.Bk;
            sn[c * Ssn + x] = st[c * Sst + g.i0 + x];
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    cluster_sync_all();  // both CTAs' barriers are initialised before any remote arrival
    const uint32_t tmem = *tmem_slot;

    auto stage_corr = [&](long long kb) {
        const Blk g = blk_of(p, kb);
        const uint32_t row = (uint32_t)q * (uint32_t)q4_of(q);
        const uint32_t bytes = (uint32_t)corr_slots(g.Bk) * row * 4u;
        mbar_expect_tx(corr_bar, bytes);
        if (bytes > 0)
            bulk_g2s(su32(base + lay.corr), p.Jc + (size_t)(kb % p.nb) * corr_slots(p.B) * row, bytes, corr_bar);
    };

    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            long long issued = 0;
            int sa = 0, lap = 0;
            bool ok = true;
            for (long long P = 0; P <= npairs && ok; ++P)
                for (int step = 0; step < 4 && ok; ++step) {
                    const Seg sg = seg_info(p, P, step, r);
                    const int r0 = sg.n > 0 ? (int)(sg.t % p.nb) * kRowsA : 0;
                    for (int k = 0; k < sg.n && ok; ++k) {
                        const int c = seg_chunk(sg, k);
                        if (lap > 0 && !mbar_wait(empty_a + 8 * sa, (uint32_t)((lap - 1) & 1), abort_flag, p.err)) {
                            ok = false;
                            break;
                        }
                        const uint32_t dst = su32(base + lay.a + sa * kSlotA), bar = full_a + 8 * sa;
                        mbar_expect_tx(bar, (uint32_t)kSlotA);
                        tma_load_3d(dst, tm_jp, 0, r0, 2 * c, bar);  // hi slab then lo slab of 128 rows
                        ++issued;
                        if (++sa == na) {
                            sa = 0;
                            ++lap;
                        }
                    }
                }
            if (*abort_flag) {
                volatile int no_abort = 0;
                for (long long u = issued > na ? issued - na : 0; u < issued; ++u)
                    mbar_wait(full_a + 8 * (int)(u % na), (uint32_t)((u / na) & 1), &no_abort, p.err);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            // kind::f16: D F32 (bit 4), A = B = F16, both K-major, N >> 3 at 17, M >> 4 at 24;
            // A (one-hot, M = 128 chains) from TMEM, B (coupling rows, N = nmma) from shared memory.
            const uint32_t idesc = (1u << 4) | ((uint32_t)(p.nmma >> 3) << 17) | ((uint32_t)(kTmNC >> 4) << 24);
            int sa = 0, sb = 0;
            uint32_t pha = 0, phb = 0;
            bool ok = true;
            for (long long P = 0; P <= npairs && ok; ++P)
                for (int step = 0; step < 4 && ok; ++step) {
                    const Seg sg = seg_info(p, P, step, r);
                    const long long j = sg.t >> 1;  // own block index
                    for (int k = 0; k < sg.n && ok; ++k) {
                        const int c = seg_chunk(sg, k);
                        const bool first = !sg.delta && c == 0;
                        if (!mbar_wait(full_b + 8 * sb, phb, abort_flag, p.err)) {
                            ok = false;
                            break;
                        }
                        if (!mbar_wait(full_a + 8 * sa, pha, abort_flag, p.err)) {
                            ok = false;
                            break;
                        }
                        if (first && j >= 2 &&
                            !mbar_wait(acc_empty + 8 * (int)(j & 1), (uint32_t)(((j - 2) >> 1) & 1), abort_flag,
                                       p.err)) {
                            ok = false;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t at = tmem + kTmOneHotCol + (uint32_t)sb * 32u;
                        const uint32_t bh = su32(base + lay.a + sa * kSlotA);
                        const uint64_t dh = desc_sw128(bh), dl = desc_sw128(bh + kTileA);
                        const uint32_t dcol = tmem + (uint32_t)(j & 1) * kTmAccCols;
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {  // +32 bytes along K = +2 in the start field
                            mma_f16_ts(dcol, at + kk * 8, dh + 2 * kk, idesc, (first && kk == 0) ? 0u : 1u);
                            mma_f16_ts(dcol, at + kk * 8, dl + 2 * kk, idesc, 1u);
                        }
                        mma_commit(empty_a + 8 * sa);
                        if (++sa == na) {
                            sa = 0;
                            pha ^= 1u;
                        }
                        mma_commit(empty_b + 8 * sb);
                        if (++sb == kTmNB) {
                            sb = 0;
                            phb ^= 1u;
                        }
                    }
                    if (ok && sg.commit_kb >= 0) mma_commit(acc_full + 8 * (int)((sg.commit_kb >> 1) & 1));
                }
        }
    } else if (warp < 6) {
        // ------------------------------------------------------------ drawers (warps 2-5)
        // Uniform control flow: every drawer runs the whole loop nest and meets
        // every named barrier; after an abort the work is skipped.
        const int w = tid - 64;                  // 0..127
        const int lane_base = 32 * (warp & 3);   // TMEM lane quarter of this warp
        const int ch = lane_base + lane;         // chain (TMEM lane) of this thread
        const int qv = q4_of(q) >> 2;            // float4s per padded coupling row
        const uint32_t st_peer = peer_addr(su32(st), (uint32_t)peer);
        const uint32_t ready_peer = peer_addr(ready, (uint32_t)peer);
        const uint64_t m = p.chain0 + cta0 + ch;
        uint32_t *const urow = reinterpret_cast<uint32_t *>(base + lay.hs) + ch * kTmUrS;
        // Ahead of own block kb (neither depends on the states): the Philox
        // numerators of its sites into this chain's row of the uniform table
        // (two independent streams at a time), and its h rows into buffer j % 2.
        auto prefetch = [&](long long kb) {
            const Blk g = blk_of(p, kb);
            const uint64_t sweep = p.sweep0 + (uint64_t)(kb / p.nb);
            for (int pp = 0; pp < g.Bk; pp += 2) {
                const uint64_t i0 = (uint64_t)(g.i0 + pp);
                const uint32_t u0 = p.sampler == BM_SAMPLER_METROPOLIS ? bm_mh_word(p.seed, m, sweep, i0, q)
                                                                      : bm_u24(p.seed, m, sweep, i0, 0);
                const uint32_t u1 = p.sampler == BM_SAMPLER_METROPOLIS ? bm_mh_word(p.seed, m, sweep, i0 + 1, q)
                                                                      : bm_u24(p.seed, m, sweep, i0 + 1, 0);
                urow[pp] = u0;
                if (pp + 1 < g.Bk) urow[pp + 1] = u1;
            }
            float *hr = hrow + ((kb >> 1) & 1) * kRowsA;
            for (int k = w; k < g.Bk * q; k += kTmDraw) hr[k] = p.h[(size_t)g.i0 * q + k];
        };
        bool ok = true;
        long long staged = 0;
        if (w == 0 && r < nblocks) {
            stage_corr(r);
            staged = 1;
        }
        if (r < nblocks) prefetch(r);
        for (long long kb = r; kb < nblocks; kb += 2) {
            const long long j = kb >> 1;
            const Blk g = blk_of(p, kb);
            const int slot = (int)(j & 1);
            const float *hr = hrow + slot * kRowsA;
            if (ok && !mbar_wait(acc_full + 8 * slot, (uint32_t)((j >> 1) & 1), abort_flag, p.err)) ok = false;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (ok && !mbar_wait(corr_bar, (uint32_t)(j & 1), abort_flag, p.err)) ok = false;
            ok = !named_bar_or(1, kTmDraw, !ok || *abort_flag);
            const uint8_t *old = snap_of(kb) + ch * Ssn;
            const uint32_t tacc = tmem + ((uint32_t)lane_base << 16) + (uint32_t)slot * kTmAccCols;
            // the fields of site pp+1 are loaded from TMEM while site pp is drawn
            // QC columns from the site's first (the ones past q belong to the
            // next site or lie past the block: masked below)
            uint32_t v[QC];
            if (ok) {
#pragma unroll
                for (int a = 0; a < QC; ++a) v[a] = tmem_ld1(tacc + (uint32_t)a);
            }
            for (int pp = 0; pp < g.Bk && ok; ++pp) {
                const int i = g.i0 + pp;
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                float H[QC];
#pragma unroll
                for (int a = 0; a < QC; ++a) {
                    asm volatile("" : "+r"(v[a]));  // not before the wait
                    H[a] = hr[pp * q + a] + __uint_as_float(v[a]);
                }
                if (pp + 1 < g.Bk) {
#pragma unroll
                    for (int a = 0; a < QC; ++a) v[a] = tmem_ld1(tacc + (uint32_t)((pp + 1) * q + a));
                }
                const uint32_t r24 = urow[pp];
                // sites jj < pp of the block redrawn since the MMAs: + J_ij(., new) - J_ij(., old)
                const float4 *cb = corr4 + (size_t)(pp * (pp - 1) / 2) * q * qv;
                for (int jj = 0; jj < pp; ++jj) {
                    const int sn = st[ch * Sst + g.i0 + jj], so = old[jj];
                    if (sn == so) continue;
                    const float4 *rn = cb + (jj * q + sn) * qv, *ro = cb + (jj * q + so) * qv;
#pragma unroll
                    for (int a4 = 0; a4 < QC / 4; ++a4) {  // past q4: the next row or the h rows, masked
                        const float4 vn = rn[a4], vo = ro[a4];
                        H[4 * a4] += vn.x - vo.x;
                        H[4 * a4 + 1] += vn.y - vo.y;
                        H[4 * a4 + 2] += vn.z - vo.z;
                        H[4 * a4 + 3] += vn.w - vo.w;
                    }
                }
#pragma unroll
                for (int a = 0; a < QC; ++a) H[a] = a < q ? H[a] * p.beta_l2e : -INFINITY;
                st[ch * Sst + i] = (uint8_t)update_symbol<QC>(H, q, st[ch * Sst + i], r24, p.sampler);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(acc_empty + 8 * slot);
            named_bar_sync(1, kTmDraw);  // the staged coupling blocks are free again
            if (w == 0 && ok && !*abort_flag && kb + 2 < nblocks) {
                stage_corr(kb + 2);
                ++staged;
            }
            // CTA 1: the next pair's snapshots, before block kb is published
            // (CTA 0 starts rewriting block kb+1's sites once it has it).
            if (r == 1 && kb + 1 < nblocks) {
                if (ok && !mbar_wait_cl(ready + 8 * (int)((kb - 1) & 1), (uint32_t)(((kb - 1) >> 1) & 1), abort_flag,
                                        p.err))
                    ok = false;
                if (ok)
                    for (long long nb2 = kb + 1; nb2 <= kb + 2 && nb2 < nblocks; ++nb2) {
                        const Blk gn = blk_of(p, nb2);
                        uint8_t *sn = snap_of(nb2) + ch * Ssn;
                        for (int x = 0; x < gn.Bk; ++x) sn[x] = st[ch * Sst + gn.i0 + x];
                    }
            }
            // Copy block kb's new states into the peer's copy.  CTA 0 first waits
            // until CTA 1's generators have finished pair j's main chunks, which
            // still read block kb's pre-redraw states from CTA 1's copy.
            if (r == 0 && ok && !mbar_wait_cl(gen_done, (uint32_t)(j & 1), abort_flag, p.err)) ok = false;
            if (ok)
                for (int x = 0; x < g.Bk; ++x)
                    st_cluster_u8(st_peer + (uint32_t)(ch * Sst + g.i0 + x), (unsigned short)st[ch * Sst + g.i0 + x]);
            // publish block kb: own generator and the peer
            mbar_arrive(ready + 8 * (int)(kb & 1));
            mbar_arrive_peer(ready_peer + 8 * (uint32_t)(kb & 1));
            if (ok && kb + 2 < nblocks) prefetch(kb + 2);
            // CTA 0: the next pair's snapshots once block kb+1 has arrived
            if (r == 0 && kb + 1 < nblocks) {
                if (ok && !mbar_wait_cl(ready + 8 * (int)((kb + 1) & 1), (uint32_t)(((kb + 1) >> 1) & 1), abort_flag,
                                        p.err))
                    ok = false;
                if (ok)
                    for (long long nb2 = kb + 2; nb2 <= kb + 3 && nb2 < nblocks; ++nb2) {
                        const Blk gn = blk_of(p, nb2);
                        uint8_t *sn = snap_of(nb2) + ch * Ssn;
                        for (int x = 0; x < gn.Bk; ++x) sn[x] = st[ch * Sst + gn.i0 + x];
                    }
                mbar_arrive(snapready);
            }
        }
        if (!ok) *abort_flag = 1;
        if (w == 0 && *abort_flag && staged > 0) {
            volatile int no_abort = 0;
            mbar_wait(corr_bar, (uint32_t)((staged - 1) & 1), &no_abort, p.err);
        }
    } else {
        // ------------------------------------------------------------ generators (warps 6-9)
        const int lane_base = 32 * (warp & 3);
        const int ch = lane_base + lane;  // operand row (TMEM lane) of chain ch
        const int st_o = (int)lay.st + ch * Sst;  // byte offsets from base: this chain's state row
        const int wrow = ch * Ssn;
        const uint32_t tone = tmem + ((uint32_t)lane_base << 16) + kTmOneHotCol;
        const uint32_t gen_done_peer = peer_addr(gen_done, (uint32_t)peer);
        int sb = 0, lap = 0;
        int pend = -1;  // ring slot whose one-hot store is still in flight
        // The previous chunk's store has completed: hand its slot to the MMA.
        auto flush = [&]() {
            if (pend >= 0) {
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(full_b + 8 * pend);
                pend = -1;
            }
        };
        bool ok = true;
        for (long long P = 0; P <= npairs && ok; ++P) {
            int s0lo = L, s0n = 0, s1lo = L, s1n = 0;  // blocks 2P-2, 2P-1: first site and size
            int ps0 = (int)lay.snap, ps1 = ps0;         // and their snapshot rows (offsets from base)
            if (P >= 1) {
                const Blk g0 = blk_of(p, 2 * P - 2), g1 = blk_of(p, 2 * P - 1);
                s0lo = g0.i0;
                s0n = g0.Bk;
                s1lo = g1.i0;
                s1n = g1.Bk;
                ps0 = (int)(snap_of(2 * P - 2) - base) + wrow;
                ps1 = (int)(snap_of(2 * P - 1) - base) + wrow;
            }
            // state of site jj as the main chunks see it (blocks being redrawn: snapshot)
            auto state = [&](int jj) {
                int o = st_o + jj;
                o = (unsigned)(jj - s0lo) < (unsigned)s0n ? ps0 + (jj - s0lo) : o;
                o = (unsigned)(jj - s1lo) < (unsigned)s1n ? ps1 + (jj - s1lo) : o;
                return (int)base[o];
            };
            for (int step = 0; step < 4 && ok; ++step) {
                const Seg sg = seg_info(p, P, step, r);
                if (sg.n > 0 && sg.wait_kind != 0) {
                    flush();  // the awaited block may need that chunk's MMAs
                    const uint32_t bar = sg.wait_kind == 1 ? ready + 8 * (uint32_t)(sg.wait_kb & 1) : snapready;
                    if (!mbar_wait_cl(bar, (uint32_t)((sg.wait_kb >> 1) & 1), abort_flag, p.err)) {
                        ok = false;
                        break;
                    }
                }
                for (int k = 0; k < sg.n; ++k) {
                    const int c = seg_chunk(sg, k);
                    const int k0 = c * kKC;
                    // bit e of (plus, minus): element k0 + e of the row is +1 / -1
                    uint32_t pl0 = 0, pl1 = 0, mi0 = 0, mi1 = 0;
                    if (!sg.delta) {
                        const int jlo = jtab[2 * c], jhi = jtab[2 * c + 1];
                        if (jhi - jlo < 8) {  // q >= 8: independent loads, no branch (sites past jhi: no bit)
#pragma unroll
                            for (int t = 0; t < 8; ++t) {
                                const int jj = min(jlo + t, jhi);
                                const int pos = jlo + t <= jhi ? jj * q + state(jj) - k0 : -1;
                                pl0 |= bit_at(pos);
                                pl1 |= bit_at(pos - 32);
                            }
                        } else {
                            for (int jj = jlo; jj <= jhi; ++jj) {
                                const int pos = jj * q + state(jj) - k0;
                                pl0 |= bit_at(pos);
                                pl1 |= bit_at(pos - 32);
                            }
                        }
                    } else {
                        for (int u = 0; u < 2; ++u) {
                            const long long db = u == 0 ? sg.d0 : sg.d1;
                            if (db < 0) continue;
                            const Blk gd = blk_of(p, db);
                            const int po = u == 0 ? ps0 : ps1;  // d0 = 2P-2, d1 = 2P-1
                            for (int x = 0; x < gd.Bk; ++x) {
                                const int jj = gd.i0 + x;
                                const int sn = base[st_o + jj], so = base[po + x];
                                if (sn == so) continue;
                                const int pn = jj * q + sn - k0, pd = jj * q + so - k0;
                                pl0 |= bit_at(pn);
                                pl1 |= bit_at(pn - 32);
                                mi0 |= bit_at(pd);
                                mi1 |= bit_at(pd - 32);
                            }
                        }
                    }
                    const uint64_t pl = ((uint64_t)pl1 << 32) | pl0, mi = ((uint64_t)mi1 << 32) | mi0;
                    if (lap > 0 && !mbar_wait(empty_b + 8 * sb, (uint32_t)((lap - 1) & 1), abort_flag, p.err)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    uint32_t v[32];
                    if (sg.delta)
                        onehot_regs<true>(pl, mi, v);
                    else
                        onehot_regs<false>(pl, 0ull, v);
                    flush();
                    tmem_st32(tone + (uint32_t)sb * 32u, v);  // completes while the next chunk is built
                    pend = sb;
                    if (++sb == kTmNB) {
                        sb = 0;
                        ++lap;
                    }
                }
                // CTA 1: pair P's main chunks are read; CTA 0 may now overwrite
                // block 2P's sites in this CTA's copy of the states
                if (ok && r == 1 && step == 2 && 2 * P < nblocks) {
                    __syncwarp();
                    if (lane == 0) mbar_arrive_peer(gen_done_peer);
                }
            }
        }
        flush();
        if (!ok) *abort_flag = 1;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmCols) : "memory");
    // No remote store or arrival into either CTA is in flight past this
    // barrier; then each CTA reads the other's abort flag, and the second
    // barrier keeps both CTAs resident until those reads are done.
    cluster_sync_all();
    const bool bad = *abort_flag != 0 || ld_cluster_u32(peer_addr(su32((const void *)abort_flag), (uint32_t)peer)) != 0;
    cluster_sync_all();
    if (bad) return;
    const int half = NC / 2;  // CTA r writes back chains 2c + r
    for (int k = tid; k < half * L; k += kTmThreads) {
        const int cc = k / L, x = k - cc * L;
        const int c = 2 * cc + r;
        const size_t mm = cta0 + c;
        if (mm < (size_t)p.M) p.states[mm * L + x] = st[c * Sst + x];
    }
}

// Jc[blk][slot][b][a4] = J_ij(a, b) for i = blk*B + pi, j = blk*B + pj,
// slot = pi*(pi-1)/2 + pj (pi > pj); zero for a >= q or i >= L.
__global__ void k_build_corr(const float *__restrict__ J, float *__restrict__ Jc, int L, int q, int B, int nb)
{
    const int q4 = q4_of(q), slots = corr_slots(B);
    const size_t n = (size_t)nb * slots * q * q4;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        const int a = (int)(t % q4);
        size_t u = t / q4;
        const int b = (int)(u % q);
        u /= q;
        const int slot = (int)(u % slots), blk = (int)(u / slots);
        int pi = 1;
        while ((pi + 1) * pi / 2 <= slot) ++pi;
        const int pj = slot - pi * (pi - 1) / 2;
        const int i = blk * B + pi, j = blk * B + pj;
        Jc[t] = (a < q && i < L) ? J[(((size_t)i * L + j) * q + a) * q + b] : 0.0f;
    }
}

int corr_prepare(bm_model_s *m, int B, cudaStream_t st)
{
    if (m->corr_current) return BM_OK;
    const int nb = (m->L + B - 1) / B;
    const size_t n = (size_t)nb * corr_slots(B) * m->q * q4_of(m->q);
    if (!m->Jc) BM_CK(cudaMalloc(&m->Jc, std::max<size_t>(n, 4) * sizeof(float)));
    if (n > 0) {
        const int grid = (int)std::min<size_t>((n + 255) / 256, 152 * 16);
        k_build_corr<<<grid, 256, 0, st>>>(m->J, m->Jc, m->L, m->q, B, nb);
        BM_CK_LAUNCH("k_build_corr");
    }
    m->corr_current = true;
    return BM_OK;
}

int g_max_clusters[64];
std::once_flag g_clusters_once[64];

// Clusters of two one-CTA-per-SM CTAs that the device runs at once.
int max_clusters(const bm_model_s *m)
{
    const int dev = m->device >= 0 && m->device < 64 ? m->device : 0;
    std::call_once(g_clusters_once[dev], [&] {
        int n = (m->num_sms > 0 ? m->num_sms : 2) / 2;
        const int smem = 200 * 1024;  // any size above half an SM's shared memory: one CTA per SM
        if (cudaFuncSetAttribute(k_gibbs_pair<false, 32, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) ==
            cudaSuccess) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(2, 1, 1);
            cfg.blockDim = dim3(kThreads, 1, 1);
            cfg.dynamicSmemBytes = smem;
            int c = 0;  // the kernel's cluster shape (2 CTAs) is fixed at compile time
            if (cudaOccupancyMaxActiveClusters(&c, k_gibbs_pair<false, 32, false>, &cfg) == cudaSuccess && c > 0) n = c;
        }
        (void)cudaGetLastError();
        g_max_clusters[dev] = n > 0 ? n : 1;
    });
    return g_max_clusters[dev];
}

// Largest chains per cluster (multiple of 16, <= min(cap, 160)) whose layout
// fits one CTA's shared memory; 0 when none does or the shape is unsupported.
int fit_nc(const bm_model_s *m, int cap, bool cg2 = false)
{
    if (m->L < 2 || m->L > 65535 || m->q > kQmax) return 0;
    const int B = bm_split_block_sites(m->L, m->q);
    if (B > kBmax) return 0;
    const int Lp = (m->L + 15) & ~15;
    const int nK = (m->L * m->q + kKC - 1) / kKC;
    int nc = std::min(cap, kNCmax) & ~15;
    while (nc >= 16 && smem_layout(nc, Lp, B, nK, m->q, cg2 ? nc / 2 : nc).total + 1024 > 227 * 1024) nc -= 16;
    return nc >= 16 ? nc : 0;
}

size_t smem_bytes(const bm_model_s *m, int nc, bool cg2 = false)
{
    const int B = bm_split_block_sites(m->L, m->q);
    return (size_t)smem_layout(nc, (m->L + 15) & ~15, B, (m->L * m->q + kKC - 1) / kKC, m->q, cg2 ? nc / 2 : nc)
               .total +
           1024;
}

void fill_args(const bm_model_s *m, const bm_chains_s *c, int NC, int nsweeps, float beta, uint8_t *states,
               PairArgs &a)
{
    a.h = m->h;
    a.Jc = m->Jc;
    a.states = states;
    a.err = m->dflags + 3;
    a.seed = c->seed;
    a.sweep0 = c->sweep;
    a.chain0 = c->chain0;
    a.beta_l2e = (float)((double)beta * 1.4426950408889634);
    a.M = c->M;
    a.L = c->L;
    a.q = c->q;
    a.Lp = (c->L + 15) & ~15;
    a.B = bm_split_block_sites(c->L, c->q);
    a.nb = (c->L + a.B - 1) / a.B;
    a.nK = m->Kp / kKC;
    a.NC = NC;
    a.nblocks = (long long)nsweeps * a.nb;
    a.X = a.nK / 2;
    a.acc_stride = NC <= 32 ? 32 : NC <= 64 ? 64 : NC <= 128 ? 128 : 256;
    a.tmem_cols = 2 * a.acc_stride;
    a.na = 0;
    a.nmma = 0;
    a.sampler = m->sampler;
}

// The shared-memory operand kernel for q rounded up to 8 (CG2: paired tensor cores).
template <bool BATCH, bool CG2 = false>
int launch_smem(int q, int grid, size_t smem, cudaStream_t st, const CUtensorMap &tm, const PairArgs &a,
                const PairItem *items)
{
    auto go = [&](auto kern) -> int {
        BM_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<grid, kThreads, smem, st>>>(tm, a, items);
        BM_CK_LAUNCH(BATCH ? "k_gibbs_pair (batch)" : CG2 ? "k_gibbs_pair (paired tensor cores)" : "k_gibbs_pair");
        return BM_OK;
    };
    switch ((q + 7) / 8) {
    case 1: return go(k_gibbs_pair<BATCH, 8, CG2>);
    case 2: return go(k_gibbs_pair<BATCH, 16, CG2>);
    case 3: return go(k_gibbs_pair<BATCH, 24, CG2>);
    default: return go(k_gibbs_pair<BATCH, 32, CG2>);
    }
}

// The tensor-memory operand kernel for q rounded up to 8.
template <bool BATCH>
int launch_tm(int q, int grid, size_t smem, cudaStream_t st, const CUtensorMap &tm, const PairArgs &a,
              const PairItem *items)
{
    auto go = [&](auto kern) -> int {
        BM_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<grid, kTmThreads, smem, st>>>(tm, a, items);
        BM_CK_LAUNCH("k_gibbs_pair_tm");
        return BM_OK;
    };
    switch ((q + 7) / 8) {
    case 1: return go(k_gibbs_pair_tm<BATCH, 8>);
    case 2: return go(k_gibbs_pair_tm<BATCH, 16>);
    case 3: return go(k_gibbs_pair_tm<BATCH, 24>);
    default: return go(k_gibbs_pair_tm<BATCH, 32>);
    }
}

// Coupling ring slots of the tensor-memory operand form for this shape (as
// many as fit one CTA's shared memory, 4 down to 2), 0 when it does not fit.
int tm_ring(const bm_model_s *m)
{
    if (m->L < 2 || m->L > 65535 || m->q > kQmax) return 0;
    const int B = bm_split_block_sites(m->L, m->q);
    if (B > kBmax || B * m->q > kRowsA) return 0;
    const int Lp = (m->L + 15) & ~15, nK = (m->L * m->q + kKC - 1) / kKC;
    for (int na = kTmNAmax; na >= 2; --na)
        if (smem_layout_tm(na, Lp, B, nK, m->q).total + 1024 <= 227 * 1024) return na;
    return 0;
}

// Ring slots when the sweep takes the tensor-memory operand form, else 0.
// That form wins where a block's draws outweigh its K chunks (measured at
// L=120 q=5 and L=64 q=21: 1.5-1.9x); where the chunks dominate (q=21,
// L >= 120) the one-hot generators set its pace and the shared-memory
// operand form is faster.
int tm_form(const bm_model_s *m)
{
    const int na = tm_ring(m);
    if (na == 0) return 0;
    const int nK = (m->L * m->q + kKC - 1) / kKC;
    return nK <= 4 * bm_split_block_sites(m->L, m->q) ? na : 0;
}

size_t smem_bytes_tm(const bm_model_s *m, int na)
{
    const int B = bm_split_block_sites(m->L, m->q);
    return (size_t)smem_layout_tm(na, (m->L + 15) & ~15, B, (m->L * m->q + kKC - 1) / kKC, m->q).total + 1024;
}

void fill_args_tm(const bm_model_s *m, const bm_chains_s *c, int na, int nsweeps, float beta, uint8_t *states,
                  PairArgs &a)
{
    fill_args(m, c, kTmNC, nsweeps, beta, states, a);
    a.na = na;
    a.nmma = (a.B * a.q + 15) & ~15;
    a.tmem_cols = kTmCols;
    a.acc_stride = kTmAccCols;
}

// The tensor-core layouts (split J, in-block corrections) of the live J.
int model_prepare(bm_model_s *m, cudaStream_t st)
{
    int rc = bm_split_prepare(m, 0, st);
    if (rc == BM_OK) rc = corr_prepare(m, bm_split_block_sites(m->L, m->q), st);
    return rc;
}

}  // namespace

int bm_corr_prepare(bm_model_s *m, cudaStream_t st)
{
    return corr_prepare(m, bm_split_block_sites(m->L, m->q), st);
}

// Chains per cluster for the two-CTA tensor-core sweep (multiple of 16,
// <= 160), or 0 when the shape does not fit one CTA's shared memory or L < 2.
int bm_gibbs_pair_chains_per_cluster(const bm_model_s *m, int M)
{
    if (tm_form(m) > 0) return kTmNC;
    const int ncl = max_clusters(m);
    const int want = std::max(16, (((M + ncl - 1) / ncl) + 15) & ~15);
    return fit_nc(m, want);
}

// True when the two-CTA sweep takes its tensor-memory operand form.
bool bm_gibbs_pair_tm(const bm_model_s *m) { return tm_form(m) > 0; }

// Waves of clusters the two-CTA sweep of M chains needs (0: does not fit).
int bm_gibbs_pair_waves(const bm_model_s *m, int M)
{
    const int nc = bm_gibbs_pair_chains_per_cluster(m, M);
    if (nc == 0) return 0;
    const int ncl = max_clusters(m);
    return ((M + nc - 1) / nc + ncl - 1) / ncl;
}

// Chains per cluster of the paired-tensor-core form (multiple of 16, <= 160),
// 0 when it does not fit.
int bm_gibbs_paired_chains_per_cluster(const bm_model_s *m, int M)
{
    const int ncl = max_clusters(m);
    const int want = std::max(16, (((M + ncl - 1) / ncl) + 15) & ~15);
    return fit_nc(m, want, true);
}

// Waves of clusters the paired-tensor-core sweep of M chains needs (0: does not fit).
int bm_gibbs_paired_waves(const bm_model_s *m, int M)
{
    const int nc = bm_gibbs_paired_chains_per_cluster(m, M);
    if (nc == 0) return 0;
    const int ncl = max_clusters(m);
    return ((M + nc - 1) / nc + ncl - 1) / ncl;
}

int bm_launch_gibbs_paired(bm_model_s *m, bm_chains_s *c, int nsweeps, float beta, cudaStream_t st)
{
    const int NC = bm_gibbs_paired_chains_per_cluster(m, c->M);
    if (NC == 0) return bm_fail(BM_EINVAL, "paired tensor-core sweep: shape does not fit shared memory");
    const int rc = model_prepare(m, st);
    if (rc != BM_OK) return rc;
    PairArgs a;
    fill_args(m, c, NC, nsweeps, beta, c->s, a);
    const size_t smem = smem_bytes(m, NC, true);
    const int nclusters = (c->M + NC - 1) / NC;
    return launch_smem<false, true>(a.q, 2 * nclusters, smem, st, *reinterpret_cast<const CUtensorMap *>(m->tmap_jp),
                                    a, nullptr);
}

int bm_launch_gibbs_pair(bm_model_s *m, bm_chains_s *c, int nsweeps, float beta, cudaStream_t st)
{
    const int NC = bm_gibbs_pair_chains_per_cluster(m, c->M);
    if (NC == 0) return bm_fail(BM_EINVAL, "two-CTA tensor-core sweep: shape does not fit shared memory");
    {
        const int rc = model_prepare(m, st);
        if (rc != BM_OK) return rc;
    }
    const int na = tm_form(m);
    if (na > 0) {
        PairArgs a;
        fill_args_tm(m, c, na, nsweeps, beta, c->s, a);
        const size_t smem = smem_bytes_tm(m, na);
        const int nclusters = (c->M + kTmNC - 1) / kTmNC;
        return launch_tm<false>(a.q, 2 * nclusters, smem, st, *reinterpret_cast<const CUtensorMap *>(m->tmap_jp), a,
                                nullptr);
    }
    PairArgs a;
    fill_args(m, c, NC, nsweeps, beta, c->s, a);
    const size_t smem = smem_bytes(m, NC);
    const int nclusters = (c->M + NC - 1) / NC;
    return launch_smem<false>(a.q, 2 * nclusters, smem, st, *reinterpret_cast<const CUtensorMap *>(m->tmap_jp), a,
                              nullptr);
}

// ---------------------------------------------------------------------------
// Batches of models: one launch, cluster k runs work item k = (model, chain
// tile), items ordered longest model first (LPT).  A model's tile size is the
// largest chain count its layout fits (fewer clusters stream its couplings),
// capped by an autotuned limit, and balanced over its tiles.
// ---------------------------------------------------------------------------
struct bm_pair_batch_s {
    std::vector<bm_model_s *> models;
    std::vector<bm_chains_s *> chains;
    int cap = kNCmax;
    std::vector<int> model_of, nc_of;
    std::vector<long long> first;
    size_t smem = 0;
    int ncmax = 0;
    PairItem *items_dev = nullptr, *items_host = nullptr;
    size_t items_cap = 0;
    cudaEvent_t used = nullptr;  // the copy of items_host made by the last launch
};

namespace {

int build_tiles(bm_pair_batch_s *b)
{
    std::vector<int> idx(b->models.size());
    for (size_t k = 0; k < idx.size(); ++k) idx[k] = (int)k;
    std::stable_sort(idx.begin(), idx.end(), [b](int x, int y) { return b->models[x]->L > b->models[y]->L; });
    b->model_of.clear();
    b->nc_of.clear();
    b->first.clear();
    b->smem = 0;
    b->ncmax = 0;
    for (int k : idx) {
        const bm_model_s *m = b->models[k];
        const int M = b->chains[k]->M;
        const int fit = fit_nc(m, b->cap);
        if (fit == 0) return bm_fail(BM_EINVAL, "batch: L=%d q=%d does not fit the tensor-core sweep", m->L, m->q);
        const int tiles = (M + fit - 1) / fit;
        const int nc = std::min(fit, (((M + tiles - 1) / tiles) + 15) & ~15);
        for (long long c0 = 0; c0 < M; c0 += nc) {
            b->model_of.push_back(k);
            b->nc_of.push_back(nc);
            b->first.push_back(c0);
        }
        b->smem = std::max(b->smem, smem_bytes(m, nc));
        b->ncmax = std::max(b->ncmax, nc);
    }
    const size_t n = b->model_of.size();
    if (n > b->items_cap) {
        if (b->used) cudaEventSynchronize(b->used);
        cudaFree(b->items_dev);
        cudaFreeHost(b->items_host);
        b->items_dev = nullptr;
        b->items_host = nullptr;
        b->items_cap = 0;
        BM_CK(cudaMalloc(&b->items_dev, n * sizeof(PairItem)));
        BM_CK(cudaMallocHost(&b->items_host, n * sizeof(PairItem)));
        b->items_cap = n;
    }
    return BM_OK;
}

}  // namespace

int bm_pair_batch_create(bm_model_s *const *models, bm_chains_s *const *chains, int count, bm_pair_batch_s **out)
{
    *out = nullptr;
    bm_pair_batch_s *b = new (std::nothrow) bm_pair_batch_s();
    if (!b) return bm_fail(BM_ENOMEM, "batch: host allocation failed");
    b->models.assign(models, models + count);
    b->chains.assign(chains, chains + count);
    int rc = build_tiles(b);
    if (rc == BM_OK && cudaEventCreateWithFlags(&b->used, cudaEventDisableTiming) != cudaSuccess)
        rc = bm_fail(BM_ECUDA, "batch: event");
    if (rc != BM_OK) {
        bm_pair_batch_free(b);
        return rc;
    }
    *out = b;
    return BM_OK;
}

void bm_pair_batch_free(bm_pair_batch_s *b)
{
    if (!b) return;
    if (b->used) {
        cudaEventSynchronize(b->used);
        cudaEventDestroy(b->used);
    }
    cudaFree(b->items_dev);
    cudaFreeHost(b->items_host);
    delete b;
}

int bm_pair_batch_sweep(bm_pair_batch_s *b, int nsweeps, float beta, cudaStream_t st, uint8_t *const *states_override)
{
    for (auto *m : b->models) {
        const int rc = model_prepare(m, st);
        if (rc != BM_OK) return rc;
    }
    const int n = (int)b->model_of.size();
    BM_CK(cudaEventSynchronize(b->used));  // the previous launch's copy of the list has been made
    for (int t = 0; t < n; ++t) {
        const int k = b->model_of[t];
        PairItem &it = b->items_host[t];
        std::memcpy(&it.tm, b->models[k]->tmap_jp, sizeof(CUtensorMap));
        fill_args(b->models[k], b->chains[k], b->nc_of[t], nsweeps, beta,
                  states_override ? states_override[k] : b->chains[k]->s, it.a);
        it.first = b->first[t];
    }
    BM_CK(cudaMemcpyAsync(b->items_dev, b->items_host, (size_t)n * sizeof(PairItem), cudaMemcpyHostToDevice, st));
    BM_CK(cudaEventRecord(b->used, st));
    return launch_smem<true>(b->models[0]->q, 2 * n, b->smem, st, b->items_host[0].tm, b->items_host[0].a,
                             b->items_dev);
}

int bm_pair_batch_autotune(bm_pair_batch_s *b, cudaStream_t st)
{
    // tuning sweeps run on scratch copies of the states: the chains do not move
    std::vector<uint8_t *> scratch(b->chains.size(), nullptr);
    int rc = BM_OK;
    for (size_t k = 0; k < b->chains.size() && rc == BM_OK; ++k) {
        const size_t n = (size_t)b->chains[k]->M * b->chains[k]->L;
        cudaError_t e = cudaMalloc(&scratch[k], n);
        if (e == cudaSuccess) e = cudaMemcpyAsync(scratch[k], b->chains[k]->s, n, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) rc = bm_cuda_fail(e, "batch autotune: scratch");
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (rc == BM_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        rc = bm_fail(BM_ECUDA, "batch autotune: events");
    int best = b->cap;
    float best_ms = 1e30f;
    for (int cap : {160, 128, 96, 64, 48, 32}) {
        if (rc != BM_OK) break;
        b->cap = cap;
        rc = build_tiles(b);
        if (rc == BM_OK) rc = bm_pair_batch_sweep(b, 1, 1.0f, st, scratch.data());  // warm-up
        if (rc == BM_OK && cudaEventRecord(e0, st) != cudaSuccess) rc = bm_fail(BM_ECUDA, "batch autotune: event");
        for (int r = 0; r < 2 && rc == BM_OK; ++r) rc = bm_pair_batch_sweep(b, 1, 1.0f, st, scratch.data());
        if (rc == BM_OK && cudaEventRecord(e1, st) != cudaSuccess) rc = bm_fail(BM_ECUDA, "batch autotune: event");
        float ms = 0.0f;
        if (rc == BM_OK &&
            (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            rc = bm_fail(BM_ECUDA, "batch autotune: timing");
        if (rc == BM_OK && ms < best_ms) {
            best_ms = ms;
            best = cap;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(st);
    for (auto *p : scratch) cudaFree(p);
    b->cap = best;
    const int rc2 = build_tiles(b);
    return rc == BM_OK ? rc2 : rc;
}

void bm_pair_batch_shape(const bm_pair_batch_s *b, int *nc, int *ctas)
{
    if (nc) *nc = b->ncmax;
    if (ctas) *ctas = 2 * (int)b->model_of.size();
}
