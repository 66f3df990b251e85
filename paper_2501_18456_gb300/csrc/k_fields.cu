// Conditional fields of a batch of sequences,
//     H[k][i][a] = h_i(a) + sum_{j != i} J_ij(a, s_j^k),
// the local field from which the Gibbs conditional of Sec. 2.1 and the
// single-mutant energies of Sec. 4.4 are formed.  Three numerical forms:
//
//   k_fields_simt      CUDA cores, FP32 sum over j ascending of the gather
//                      rows Jg[i][j][s_j][.] (J_ii = 0 contributes 0);
//   k_fields_tc<T>     tensor cores: G = J . X^T with X the one-hot of the
//                      sequences, J split as T hi + T lo (T = fp16 or bf16,
//                      round to nearest) and both parts accumulated in FP32
//                      in TMEM; H = h + G.
//
// k_fields_tc is persistent over output tiles of 128 rows (i,a) (one padded
// site block of the split layout) x 256 sequences.  warp 0 streams per
// 64-column K chunk the hi and lo coupling tiles (two 16 KB TMA copies) and
// the one-hot tile of the 256 sequences (one 32 KB copy, 128B swizzle) into a
// 3-stage ring; warp 1 issues 8 MMAs per chunk (kind::f16, M = 128,
// N = 256, K = 16, hi then lo) into one of two TMEM accumulators; warps 2-5
// add h and store H (one TMEM lane = one row (i,a), so a warp's stores are
// contiguous) while the next tile accumulates.  A symbol >= q contributes
// nothing in either form and is flagged.
#include "bm_internal.cuh"
#include "tc_common.cuh"

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>

namespace {

using namespace bmtc;

// ---------------------------------------------------------------------------
// FP32 CUDA-core form: one block per sequence (grid-stride), thread per (i,a).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_fields_simt(const float *__restrict__ h, const float *__restrict__ Jg, int bs,
                                                     int L, int q, const uint8_t *__restrict__ S, int n,
                                                     float *__restrict__ H, int *bad)
{
    extern __shared__ uint8_t sv[];
    const int Q = L * q;
    for (long long k = blockIdx.x; k < n; k += gridDim.x) {
        __syncthreads();  // sv of the previous sequence is no longer read
        int inval = 0;
        for (int t = threadIdx.x; t < L; t += blockDim.x) {
            const uint8_t v = S[(size_t)k * L + t];
            inval |= v >= q;
            sv[t] = v;
        }
        if (__syncthreads_or(inval) && threadIdx.x == 0) atomicOr(bad, 1);
        for (int o = threadIdx.x; o < Q; o += blockDim.x) {
            const int i = o / q, a = o - i * q;
            const float *row = Jg + (size_t)i * L * bs + a;
            float acc = 0.0f;
            for (int j = 0; j < L; ++j) {
                const int sj = sv[j];
                if (sj < q) acc += __ldg(row + (size_t)j * bs + sj * q);
            }
            H[(size_t)k * Q + o] = h[o] + acc;
        }
    }
}

// ---------------------------------------------------------------------------
// Tensor-core form.
// ---------------------------------------------------------------------------
constexpr int kKC = 64;                  // K columns per chunk (128-byte rows)
constexpr int kRows = 128;               // MMA M: rows (i,a) of a padded site block
constexpr int kCols = 256;               // MMA N: sequences per tile
constexpr int kTileA = kRows * 128;      // 16 KB (hi or lo)
constexpr int kTileB = kCols * 128;      // 32 KB
constexpr int kStage = 2 * kTileA + kTileB;
constexpr int kNS = 3;
constexpr int kThreads = 192;

__device__ __forceinline__ uint32_t one_bits(__half *) { return 0x3c00u; }
__device__ __forceinline__ uint32_t one_bits(__nv_bfloat16 *) { return 0x3f80u; }

// X[k][c] = 1 (T) if c = j*q + s_j^k for some site j with s_j^k < q, else 0;
// Kp columns.  One thread writes one 16-byte piece (8 columns).
template <typename T>
__global__ void k_onehot_rows(const uint8_t *__restrict__ S, int n, int L, int q, int Kp, T *__restrict__ X)
{
    const uint32_t one = one_bits((T *)nullptr);
    const size_t npieces = (size_t)n * (Kp / 8);
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < npieces; t += (size_t)gridDim.x * blockDim.x) {
        const size_t k = t / (Kp / 8);
        const int c0 = (int)(t - k * (Kp / 8)) * 8;
        uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int c = c0 + e, j = c / q, b = c - j * q;
            if (j < L && S[k * L + j] == b) w[e >> 1] |= one << (16 * (e & 1));
        }
        *reinterpret_cast<uint4 *>(X + k * Kp + c0) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

struct FtArgs {
    const float *h;
    float *H;
    int *err;
    int L, q, B, nb, nK, n, ntiles;
    uint32_t idesc;
};

__global__ void __launch_bounds__(kThreads, 1) k_fields_tc(const __grid_constant__ CUtensorMap tm_j,
                                                           const __grid_constant__ CUtensorMap tm_x, const FtArgs p)
{
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = su32(smem_raw);
    unsigned char *base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + kNS * kStage);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * kNS + 5);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const uint32_t full = su32(bars), empty = full + 8 * kNS;
    const uint32_t acc_full = empty + 8 * kNS, acc_empty = acc_full + 16, fin = acc_empty + 16;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = p.q, L = p.L, Q = L * q;

    if (tid == 0) {
        for (int s = 0; s < kNS; ++s) {
            mbar_init(full + 8 * s, 1);
            mbar_init(empty + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(acc_full + 8 * b, 1);
            mbar_init(acc_empty + 8 * b, 4);
        }
        mbar_init(fin, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(2 * kCols)
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
                const int rb = t % p.nb, nt = t / p.nb;
                for (int c = 0; c < p.nK; ++c) {
                    if (lap > 0 && !mbar_wait(empty + 8 * s, (uint32_t)((lap - 1) & 1), abort_flag, p.err)) {
                        ok = false;
                        break;
                    }
                    const uint32_t dst = su32(base + s * kStage), bar = full + 8 * s;
                    mbar_expect_tx(bar, kStage);
                    tma_load_3d(dst, &tm_j, 0, rb * kRows, 2 * c, bar);               // hi
                    tma_load_3d(dst + kTileA, &tm_j, 0, rb * kRows, 2 * c + 1, bar);  // lo
                    tma_load_2d(dst + 2 * kTileA, &tm_x, c * kKC, nt * kCols, bar);    // one-hot
                    ++issued;
                    if (++s == kNS) {
                        s = 0;
                        ++lap;
                    }
                }
            }
            if (*abort_flag) {
                volatile int no_abort = 0;
                for (long long u = issued > kNS ? issued - kNS : 0; u < issued; ++u)
                    mbar_wait(full + 8 * (int)(u % kNS), (uint32_t)((u / kNS) & 1), &no_abort, p.err);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            int s = 0, n = 0;
            uint32_t ph = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < p.ntiles && ok; t += gridDim.x, ++n) {
                const int buf = n & 1;
                if (n >= 2 && !mbar_wait(acc_empty + 8 * buf, (uint32_t)(((n - 2) >> 1) & 1), abort_flag, p.err)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t dcol = tmem + (uint32_t)buf * kCols;
                for (int c = 0; c < p.nK; ++c) {
                    if (!mbar_wait(full + 8 * s, ph, abort_flag, p.err)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t ah = su32(base + s * kStage), al = ah + kTileA, bx = ah + 2 * kTileA;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint64_t bd = desc_sw128(bx + kk * 32);
                        mma_f16(dcol, desc_sw128(ah + kk * 32), bd, p.idesc, (c > 0 || kk > 0) ? 1u : 0u);
                        mma_f16(dcol, desc_sw128(al + kk * 32), bd, p.idesc, 1u);
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
            mma_commit(fin);  // every MMA retired before TMEM is released
            volatile int no_abort = 0;
            mbar_wait(fin, 0, &no_abort, p.err);
        }
    } else {
        // ------------------------------------------------------------ epilogue (warps 2-5)
        const int lane_base = 32 * (warp & 3);
        const int r = lane_base + lane;  // TMEM lane = row (i,a) of the block
        const int pp = r / q, a = r - pp * q;
        int n = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < p.ntiles; t += gridDim.x, ++n) {
            const int rb = t % p.nb, nt = t / p.nb;
            const int buf = n & 1;
            if (ok && !mbar_wait(acc_full + 8 * buf, (uint32_t)((n >> 1) & 1), abort_flag, p.err)) ok = false;
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int i = rb * p.B + pp;
            const bool row_ok = pp < p.B && i < L;
            const float hv = row_ok ? p.h[i * q + a] : 0.0f;
            for (int c0 = 0; c0 < kCols; c0 += 32) {
                uint32_t v[32];
                tmem_ld32(tmem + ((uint32_t)lane_base << 16) + (uint32_t)buf * kCols + (uint32_t)c0, v);
                if (!row_ok) continue;
#pragma unroll
                for (int e = 0; e < 32; ++e) {
                    const int k = nt * kCols + c0 + e;
                    if (k < p.n) p.H[(size_t)k * Q + i * q + a] = hv + __uint_as_float(v[e]);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(acc_empty + 8 * buf);
        }
        if (!ok) *abort_flag = 1;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kCols) : "memory");
}

// Flags sequences holding a symbol >= q (they contribute nothing).
__global__ void k_flag_symbols(const uint8_t *__restrict__ S, size_t count, int q, int *bad)
{
    int inval = 0;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (size_t)gridDim.x * blockDim.x)
        inval |= S[t] >= q;
    if (__syncthreads_or(inval) && threadIdx.x == 0) atomicOr(bad, 1);
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

}  // namespace

int bm_launch_fields_simt(const bm_model_s *m, const uint8_t *seqs, int n, float *H, cudaStream_t st)
{
    if (n == 0) return BM_OK;
    const int grid = std::min(n, 152 * 8);
    k_fields_simt<<<grid, 256, (size_t)m->L, st>>>(m->h, m->Jg, m->bs, m->L, m->q, seqs, n, H, m->dflags + 4);
    BM_CK_LAUNCH("k_fields_simt");
    return BM_OK;
}

int bm_launch_fields_tc(bm_model_s *m, const uint8_t *seqs, int n, float *H, int bf16, cudaStream_t st)
{
    if (n == 0) return BM_OK;
    int rc = bm_split_prepare(m, bf16, st);
    if (rc != BM_OK) return rc;
    const int L = m->L, q = m->q, Kp = m->Kp;
    const int B = bm_split_block_sites(L, q), nb = (L + B - 1) / B;
    EncodeTiledFn fn = encode_fn();
    if (!fn) return bm_fail(BM_ECUDA, "cuTensorMapEncodeTiled entry point unavailable");

    // one-hot of the sequences, [nbatch][Kp] 16-bit, in batches of at most kBatch sequences
    constexpr int kBatch = 1 << 16;
    const int nbuf = std::min(n, kBatch);
    void *X = nullptr;
    BM_CK(cudaMallocAsync(&X, (size_t)nbuf * Kp * 2, st));
    cudaError_t e = cudaSuccess;
    {
        const size_t count = (size_t)n * L;
        k_flag_symbols<<<(int)std::min<size_t>((count + 255) / 256, 152 * 16), 256, 0, st>>>(seqs, count, q,
                                                                                        m->dflags + 4);
        e = cudaGetLastError();
    }
    const size_t smem = (size_t)kNS * kStage + (2 * kNS + 5) * 8 + 16 + 1024;
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fields_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    for (int k0 = 0; k0 < n && e == cudaSuccess && rc == BM_OK; k0 += kBatch) {
        const int nb_seq = std::min(kBatch, n - k0);
        const uint8_t *S = seqs + (size_t)k0 * L;
        const size_t npieces = (size_t)nb_seq * (Kp / 8);
        const int g1 = (int)std::min<size_t>((npieces + 255) / 256, 152 * 32);
        if (bf16)
            k_onehot_rows<__nv_bfloat16><<<g1, 256, 0, st>>>(S, nb_seq, L, q, Kp, (__nv_bfloat16 *)X);
        else
            k_onehot_rows<__half><<<g1, 256, 0, st>>>(S, nb_seq, L, q, Kp, (__half *)X);
        e = cudaGetLastError();
        if (e != cudaSuccess) break;
        alignas(64) CUtensorMap tmx;
        cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)nb_seq};
        cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
        cuuint32_t box[2] = {(cuuint32_t)kKC, (cuuint32_t)kCols};
        cuuint32_t estr[2] = {1, 1};
        const CUresult r = fn(&tmx, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, X,
                              dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            rc = bm_fail(BM_ECUDA, "cuTensorMapEncodeTiled (fields one-hot) failed (%d)", (int)r);
            break;
        }
        FtArgs a;
        a.h = m->h;
        a.H = H + (size_t)k0 * L * q;
        a.err = m->dflags + 3;
        a.L = L;
        a.q = q;
        a.B = B;
        a.nb = nb;
        a.nK = Kp / kKC;
        a.n = nb_seq;
        a.ntiles = nb * ((nb_seq + kCols - 1) / kCols);
        // kind::f16: D F32 (bit 4), A = B = fp16 (0) or bf16 (1) at bits 7 and 10, N >> 3 at 17, M >> 4 at 24.
        const uint32_t fmt = bf16 ? 1u : 0u;
        a.idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kCols >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);
        const int nsm = m->num_sms > 0 ? m->num_sms : 1;
        const int grid = std::min(a.ntiles, nsm);
        const CUtensorMap *tj = reinterpret_cast<const CUtensorMap *>(bf16 ? m->tmap_bf1 : m->tmap_j1);
        k_fields_tc<<<grid, kThreads, smem, st>>>(*tj, tmx, a);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess && rc == BM_OK) rc = bm_cuda_fail(e, "k_fields_tc");
    cudaFreeAsync(X, st);
    return rc;
}
