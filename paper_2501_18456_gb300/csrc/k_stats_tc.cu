// Chain pair counts as a TMA-fed tensor-core product (tcgen05 + TMEM + TMA).
//
// The model statistics of Sec. 2.1 are the counts
//     C[(i,a),(j,b)] = #{m : s_i^m = a, s_j^m = b} = (X^T X)[(i,a),(j,b)],
// X the one-hot encoding of the chains, X[m][(i,a)] = [s_i^m == a].  This is
// a dense contraction over the chain index with exact 0/1 operands; FP8 E4M3
// (1.0 = 0x38) operands with FP32 accumulation give exact counts below 2^24.
//
// Two kernels:
//   k_onehot_t   writes X^T once per call: XT[(i,a)][m] (Q = L*q rows, Mp
//                chain columns, zero padded to a multiple of 256), coalesced
//                16-byte stores from a shared-memory transpose of the states;
//   k_counts_tc  persistent over the output tiles that hold some pair i <= j.
//                A tile is 256 rows (i,a) x 256 columns (j,b), T = floor(256/q)
//                sites each way.  warp 0 streams the A (256 rows) and B (256
//                rows) operand tiles of 128 chains per stage by TMA (3-D
//                view, 128B swizzle) into a 3-stage ring; warp 1 issues 8 MMAs
//                per stage (kind::f8f6f4, M = 128, N = 256, K = 32: each B
//                tile feeds the two 128-row halves of A) into two TMEM
//                accumulators (512 columns); warps 2-9 read them (one TMEM
//                lane = one row) and store the int32 counts of the blocks
//                i <= j in the upper block-triangle layout.
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

constexpr int kTile = 256;           // output tile: 256 rows (i,a) x 256 columns (j,b)
constexpr int kHalf = 128;           // MMA M: one accumulator per 128-row half of the tile
constexpr int kKB = 128;             // chains per stage (one 128-byte swizzle atom per row)
constexpr int kKS = 1;               // atoms per stage
constexpr int kStageA = kTile * kKB; // 32 KB
constexpr int kStageB = kTile * kKB; // 32 KB
constexpr int kNS = 3;               // stages
constexpr int kThreads = 320;        // 10 warps: producer, MMA issuer, 8 epilogue warps
constexpr int kStgStride = 33;       // staging row stride (floats): conflict-free both ways

// ---------------------------------------------------------------------------
// X^T, E4M3 one-hot.  Block: 128 chains x 32 sites, 256 threads.
// ---------------------------------------------------------------------------
constexpr int kOtChains = 128, kOtSites = 32;

__global__ void __launch_bounds__(256) k_onehot_t(const uint8_t *__restrict__ S, int M, int L, int q, int Mp,
                                                  uint8_t *__restrict__ XT)
{
    __shared__ uint8_t sv[kOtSites][kOtChains + 4];  // states transposed: [site][chain]
    const int m0 = blockIdx.x * kOtChains, i0 = blockIdx.y * kOtSites;
    const int ns = min(kOtSites, L - i0);
    for (int k = threadIdx.x; k < kOtChains * kOtSites; k += blockDim.x) {
        const int c = k / kOtSites, x = k - c * kOtSites;  // consecutive threads: consecutive sites of a chain
        const int m = m0 + c;
        sv[x][c] = (m < M && x < ns) ? S[(size_t)m * L + i0 + x] : (uint8_t)0xff;  // 0xff: padding chain
    }
    __syncthreads();
    // rows (i,a) of this site range, 8 segments of 16 chains each
    const int nrow = ns * q;
    for (int k = threadIdx.x; k < nrow * 8; k += blockDim.x) {
        const int r = k >> 3, seg = k & 7;
        const int x = r / q, a = r - x * q;
        const uint8_t *src = &sv[x][seg * 16];
        uint32_t w[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            uint32_t v = 0;
#pragma unroll
            for (int b = 0; b < 4; ++b) v |= (src[4 * u + b] == a ? 0x38u : 0u) << (8 * b);
            w[u] = v;
        }
        const size_t row = (size_t)(i0 + x) * q + a;
        *reinterpret_cast<uint4 *>(XT + row * Mp + m0 + seg * 16) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// ---------------------------------------------------------------------------
// Persistent counts GEMM.
// ---------------------------------------------------------------------------
struct CtArgs {
    int32_t *counts;
    int *err;
    int L, q, TI, TJ, nti, ntj, ntiles, nstages;  // nstages: K stages (256 chains each) per tile
};

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

__global__ void __launch_bounds__(kThreads, 1) k_counts_tc(const __grid_constant__ CUtensorMap tm_x, const CtArgs p)
{
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = su32(smem_raw);
    unsigned char *base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    // stage s: A (256 rows) at s*(kStageA + kStageB), B (256 rows) right after;
    // then the epilogue's staging of one 32-column slab of the tile
    float *stg = reinterpret_cast<float *>(base + kNS * (kStageA + kStageB));
    uint64_t *bars = reinterpret_cast<uint64_t *>(stg + kTile * kStgStride);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * kNS + 3);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const uint32_t full = su32(bars), empty = full + 8 * kNS;
    const uint32_t acc_full = empty + 8 * kNS, acc_empty = acc_full + 8;
    const uint32_t fin = acc_empty + 8;  // completion of every MMA issued (teardown)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = p.q, L = p.L;

    if (tid == 0) {
        for (int s = 0; s < kNS; ++s) {
            mbar_init(full + 8 * s, 1);
            mbar_init(empty + 8 * s, 1);
        }
        mbar_init(acc_full, 1);
        mbar_init(acc_empty, 8);
        mbar_init(fin, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(2 * kTile)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            int s = 0, lap = 0;
            long long issued = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < p.ntiles && ok; t += gridDim.x) {
                int ti, tj;
                tile_of(p, t, ti, tj);
                for (int k = 0; k < p.nstages; ++k) {
                    if (lap > 0 && !mbar_wait(empty + 8 * s, (uint32_t)((lap - 1) & 1), abort_flag, p.err)) {
                        ok = false;
                        break;
                    }
                    const uint32_t dst = su32(base + s * (kStageA + kStageB));
                    mbar_expect_tx(full + 8 * s, kStageA + kStageB);
                    tma_load_3d(dst, &tm_x, 0, ti * p.TI * q, k, full + 8 * s);
                    tma_load_3d(dst + kStageA, &tm_x, 0, tj * p.TJ * q, k, full + 8 * s);
                    ++issued;
                    if (++s == kNS) {
                        s = 0;
                        ++lap;
                    }
                }
            }
            if (*abort_flag) {  // let the copies in flight land before exit
                volatile int no_abort = 0;
                for (long long u = issued > kNS ? issued - kNS : 0; u < issued; ++u)
                    mbar_wait(full + 8 * (int)(u % kNS), (uint32_t)((u / kNS) & 1), &no_abort, p.err);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            // kind::f8f6f4: D F32 (bit 4), A = B = E4M3 (0), K-major, N >> 3 at 17, M >> 4 at 24.
            const uint32_t idesc = (1u << 4) | ((uint32_t)(kTile >> 3) << 17) | ((uint32_t)(kHalf >> 4) << 24);
            int s = 0;
            uint32_t ph = 0;
            int n = 0;  // tiles done by this CTA
            bool ok = true;
            for (int t = blockIdx.x; t < p.ntiles && ok; t += gridDim.x, ++n) {
                if (n >= 1 && !mbar_wait(acc_empty, (uint32_t)((n - 1) & 1), abort_flag, p.err)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                for (int k = 0; k < p.nstages; ++k) {
                    if (!mbar_wait(full + 8 * s, ph, abort_flag, p.err)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t a0 = su32(base + s * (kStageA + kStageB)), b0 = a0 + kStageA;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint64_t bd = desc_sw128(b0 + kk * 32);
                        const uint32_t acc = (k > 0 || kk > 0) ? 1u : 0u;
                        mma_f8(tmem, desc_sw128(a0 + kk * 32), bd, idesc, acc);                       // rows 0-127
                        mma_f8(tmem + kTile, desc_sw128(a0 + kHalf * kKB + kk * 32), bd, idesc, acc);  // rows 128-255
                    }
                    mma_commit(empty + 8 * s);
                    if (++s == kNS) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
                if (!ok) break;
                mma_commit(acc_full);
            }
            // all MMAs of this thread retired before TMEM is released (also after an abort)
            mma_commit(fin);
            volatile int no_abort = 0;
            mbar_wait(fin, 0, &no_abort, p.err);
        }
    } else {
        // ------------------------------------------------------------ epilogue (warps 2-9)
        // Per 32-column slab: each warp copies its 32 accumulator rows to the
        // staging buffer (one row per lane), then the 256 threads write the
        // slab out row by row, 32 consecutive columns per warp, so a store
        // covers a contiguous run of a block row.  Uniform control flow (the
        // named barriers) also after an abort.
        const int half = (warp - 2) >> 2;  // accumulator: tile rows [128*half, 128*half + 128)
        const int lane_base = 32 * (warp & 3);
        const int r = half * kHalf + lane_base + lane;  // tile row copied by this thread
        const int e = tid - 64;                          // 0..255
        int n = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < p.ntiles; t += gridDim.x, ++n) {
            int ti, tj;
            tile_of(p, t, ti, tj);
            if (ok && !mbar_wait(acc_full, (uint32_t)(n & 1), abort_flag, p.err)) ok = false;
            if (named_bar_or(1, 256, !ok || *abort_flag)) {  // the same decision in every epilogue thread
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int c0 = 0; c0 < kTile; c0 += 32) {
                uint32_t v[32];
                tmem_ld32(tmem + ((uint32_t)lane_base << 16) + (uint32_t)half * kTile + (uint32_t)c0, v);
#pragma unroll
                for (int x = 0; x < 32; ++x) stg[r * kStgStride + x] = __uint_as_float(v[x]);
                named_bar_sync(1, 256);
                // write-out: thread e handles column c0 + (e & 31) of rows e/32, e/32 + 8, ...
                const int cc = c0 + (e & 31);
                const int jl = cc / q, b = cc - jl * q;
                const int j = tj * p.TJ + jl;
                if (jl < p.TJ && j < L) {
                    for (int rr = e >> 5; rr < kTile; rr += 8) {
                        const int il = rr / q, a = rr - il * q;
                        const int i = ti * p.TI + il;
                        if (il < p.TI && i <= j)
                            p.counts[bm_pair_block(L, i, j) * q * q + (size_t)a * q + b] =
                                (int32_t)stg[rr * kStgStride + (e & 31)];
                    }
                }
                named_bar_sync(1, 256);  // staging is rewritten by the next slab
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(acc_empty);
        }
        if (!ok) *abort_flag = 1;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kTile) : "memory");
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
// box {128, rows, kKS}: kKS consecutive 128-chain atoms of `rows` rows.
int make_xt_map(CUtensorMap *map, const uint8_t *xt, int Q, int Mp, int rows)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return bm_fail(BM_ECUDA, "cuTensorMapEncodeTiled entry point unavailable");
    cuuint64_t dims[3] = {(cuuint64_t)kKB, (cuuint64_t)Q, (cuuint64_t)(Mp / kKB)};
    cuuint64_t strides[2] = {(cuuint64_t)Mp, (cuuint64_t)kKB};
    cuuint32_t box[3] = {(cuuint32_t)kKB, (cuuint32_t)rows, (cuuint32_t)kKS};
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
    const int Mp = (M + 255) / 256 * 256;  // chains zero padded (a multiple of the 128-chain stage)
    const size_t bytes = (size_t)Q * Mp;
    if (!c->xt || c->xt_rows != Q || c->xt_cols != Mp) {
        if (c->xt) cudaFree(c->xt);
        c->xt = nullptr;
        BM_CK(cudaMalloc(&c->xt, bytes));
        c->xt_rows = Q;
        c->xt_cols = Mp;
        const int rc = make_xt_map(reinterpret_cast<CUtensorMap *>(c->tmap_a), (const uint8_t *)c->xt, Q, Mp, kTile);
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
    a.nstages = Mp / (kKB * kKS);
    int dev = 0, nsm = 0;
    BM_CK(cudaGetDevice(&dev));
    BM_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const size_t smem = (size_t)kNS * (kStageA + kStageB) + (size_t)kTile * kStgStride * 4 + (2 * kNS + 3) * 8 + 16 + 1024;
    BM_CK(cudaFuncSetAttribute(k_counts_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = std::min(a.ntiles, nsm);
    k_counts_tc<<<grid, kThreads, smem, st>>>(*reinterpret_cast<const CUtensorMap *>(c->tmap_a), a);
    BM_CK_LAUNCH("k_counts_tc");
    return BM_OK;
}
