// Frequency statistics: chain pair counts, importance weights and weighted
// data frequencies.
//
//   chain counts   (Sec. 2.1, p_i and p_ij as chain frequencies)
//   weights        (Eq. 7, identity >= threshold, w = 1/N_m; M_eff Sec. 3.3)
//   data stats     (Eq. 3 with the pseudocount of Eqs. 8-9)
//
// All three are histogram / counting problems over a few MB of uint8
// states, so they run on CUDA cores with shared-memory histograms; every
// sum is integer (or 64-bit fixed point for weights), hence deterministic.
#include "bm_internal.cuh"

#include <algorithm>

namespace {

// ----------------------------------------------------------------------------
// Pair tiles: the L sites are cut into tiles of TS sites; the CTA for tile
// pair (ti <= tj) owns the TS x TS site pairs of that tile pair and keeps
// one q x q histogram per site pair in shared memory.  Items are
// (sequence, site pair); lanes of a warp take different site pairs of the
// same sequence so that their atomics hit different histograms.
// ----------------------------------------------------------------------------
__device__ __forceinline__ void tile_pair_from_index(int t, int nt, int &ti, int &tj)
{
    // Row-major enumeration of the upper triangle of an nt x nt grid.
    int r = 0, rem = t;
    while (rem >= nt - r) { rem -= nt - r; ++r; }
    ti = r;
    tj = r + rem;
}

constexpr int kChunk = 256;  // sequences staged per round

template <int TS>
__global__ void __launch_bounds__(512) k_chain_pairs(const uint8_t *__restrict__ S, int M, int L,
                                                     int q, int nt, int32_t *__restrict__ counts)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int *hist = reinterpret_cast<int *>(smem_raw);                      // TS*TS*q*q
    const int qq = q * q;
    uint8_t *st = reinterpret_cast<uint8_t *>(hist + TS * TS * qq);     // kChunk x 2TS
    int ti, tj;
    tile_pair_from_index(blockIdx.x, nt, ti, tj);
    const int i0 = ti * TS, j0 = tj * TS;
    for (int k = threadIdx.x; k < TS * TS * qq; k += blockDim.x) hist[k] = 0;

    for (int c0 = 0; c0 < M; c0 += kChunk) {
        const int nc = min(kChunk, M - c0);
        __syncthreads();
        for (int k = threadIdx.x; k < nc * 2 * TS; k += blockDim.x) {
            const int c = k / (2 * TS), x = k % (2 * TS);
            const int site = x < TS ? i0 + x : j0 + (x - TS);
            st[k] = site < L ? S[(size_t)(c0 + c) * L + site] : 0;
        }
        __syncthreads();
        const int items = nc * TS * TS;
        for (int it = threadIdx.x; it < items; it += blockDim.x) {
            const int c = it / (TS * TS), p = it % (TS * TS);
            const int ii = p / TS, jj = p % TS;
            const int a = st[c * 2 * TS + ii], b = st[c * 2 * TS + TS + jj];
            atomicAdd(&hist[p * qq + a * q + b], 1);
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < TS * TS * qq; k += blockDim.x) {
        const int p = k / qq, e = k % qq;
        const int i = i0 + p / TS, j = j0 + p % TS;
        if (i < L && j < L && i <= j) counts[bm_pair_block(L, i, j) * qq + e] = hist[k];
    }
}

// ----------------------------------------------------------------------------
// Weighted data pairs in 64-bit fixed point (weight * 2^40, rounded).
// ----------------------------------------------------------------------------

template <int TS>
__global__ void __launch_bounds__(512) k_data_pairs(const uint8_t *__restrict__ X,
                                                    const float *__restrict__ w, int N, int L,
                                                    int q, int nt, double meff, double alpha,
                                                    float *__restrict__ fi,
                                                    float *__restrict__ fij)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int qq = q * q;
    unsigned long long *hist = reinterpret_cast<unsigned long long *>(smem_raw);  // TS*TS*qq
    unsigned long long *wf = hist + TS * TS * qq;                                  // kChunk
    uint8_t *st = reinterpret_cast<uint8_t *>(wf + kChunk);                        // kChunk x 2TS
    int ti, tj;
    tile_pair_from_index(blockIdx.x, nt, ti, tj);
    const int i0 = ti * TS, j0 = tj * TS;
    for (int k = threadIdx.x; k < TS * TS * qq; k += blockDim.x) hist[k] = 0ull;

    for (int c0 = 0; c0 < N; c0 += kChunk) {
        const int nc = min(kChunk, N - c0);
        __syncthreads();
        for (int k = threadIdx.x; k < nc * 2 * TS; k += blockDim.x) {
            const int c = k / (2 * TS), x = k % (2 * TS);
            const int site = x < TS ? i0 + x : j0 + (x - TS);
            st[k] = site < L ? X[(size_t)(c0 + c) * L + site] : 0;
        }
        for (int k = threadIdx.x; k < nc; k += blockDim.x) {
            const double wv = w ? (double)w[c0 + k] : 1.0;
            wf[k] = (unsigned long long)llrint(wv * 1099511627776.0);  // * 2^40
        }
        __syncthreads();
        const int items = nc * TS * TS;
        for (int it = threadIdx.x; it < items; it += blockDim.x) {
            const int c = it / (TS * TS), p = it % (TS * TS);
            const int ii = p / TS, jj = p % TS;
            const int a = st[c * 2 * TS + ii], b = st[c * 2 * TS + TS + jj];
            atomicAdd(&hist[p * qq + a * q + b], wf[c]);
        }
    }
    __syncthreads();
    const double scale = (1.0 - alpha) / (meff * 1099511627776.0);
    const double pc2 = alpha / ((double)q * q), pc1 = alpha / q;
    for (int k = threadIdx.x; k < TS * TS * qq; k += blockDim.x) {
        const int p = k / qq, e = k % qq;
        const int i = i0 + p / TS, j = j0 + p % TS;
        if (i >= L || j >= L || i > j) continue;
        const int a = e / q, b = e % q;
        const double raw = (double)hist[k] * scale;
        if (i < j) {
            const float f = (float)(raw + pc2);
            fij[(((size_t)i * L + j) * q + a) * q + b] = f;
            fij[(((size_t)j * L + i) * q + b) * q + a] = f;
        } else {
            // Diagonal block: f_ii(a,b) = delta_ab f_i(a).
            const float f1 = (float)(raw + pc1);
            fij[(((size_t)i * L + i) * q + a) * q + b] = (a == b) ? f1 : 0.0f;
            if (a == b) fi[(size_t)i * q + a] = f1;
        }
    }
}

// ----------------------------------------------------------------------------
// Sum / max / min of weights (FP64, deterministic two-stage in one CTA).
// ----------------------------------------------------------------------------
__global__ void k_weight_sum(const float *__restrict__ w, int N, double *out3)
{
    __shared__ double ssum[1024], smax[1024], smin[1024];
    double s = 0.0, mx = -INFINITY, mn = INFINITY;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const double v = (double)w[k];
        s += v;
        mx = fmax(mx, v);
        mn = fmin(mn, v);
        if (!isfinite(v)) mx = INFINITY;  // non-finite weights surface as +inf max
    }
    ssum[threadIdx.x] = s;
    smax[threadIdx.x] = mx;
    smin[threadIdx.x] = mn;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            ssum[threadIdx.x] += ssum[threadIdx.x + o];
            smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + o]);
            smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out3[0] = ssum[0];
        out3[1] = smax[0];
        out3[2] = smin[0];
    }
}

// ----------------------------------------------------------------------------
// Sequence identity counts for the weights (Eq. 7).  Rows are compared four
// symbols per 32-bit word: x = a ^ b has a zero byte exactly where the
// symbols agree; ((x & 0x7f7f7f7f) + 0x7f7f7f7f) | x has bit 7 clear exactly
// in those bytes, so ~that & 0x80808080 marks the matches.  Per-byte match
// counters are accumulated in one word (at most 64 words per chunk, so no
// byte overflows) and folded at the end of each chunk.
// Tiles of 64 x 64 sequences; only tiles tm <= tn are visited and each
// qualifying pair credits both of its sequences.
// ----------------------------------------------------------------------------
constexpr int kWT = 64;      // sequences per tile side
constexpr int kWChunk = 64;  // 32-bit words per L chunk (256 symbols)

__device__ __forceinline__ uint32_t match_bytes(uint32_t a, uint32_t b)
{
    const uint32_t x = a ^ b;
    const uint32_t t = ((x & 0x7f7f7f7fu) + 0x7f7f7f7fu) | x;
    return (~t & 0x80808080u) >> 7;  // 1 in every byte where a and b agree
}

__device__ __forceinline__ int fold_bytes(uint32_t v)
{
    const uint32_t p = (v & 0x00ff00ffu) + ((v >> 8) & 0x00ff00ffu);
    return (int)((p & 0xffffu) + (p >> 16));
}

__global__ void __launch_bounds__(256) k_identity(const uint8_t *__restrict__ X, int N, int L,
                                                  int thr, int ntile, int *__restrict__ cnt)
{
    __shared__ uint32_t A[kWT][kWChunk + 1];
    __shared__ uint32_t B[kWT][kWChunk + 1];
    __shared__ int cntA[kWT], cntB[kWT];
    int tm, tn;
    tile_pair_from_index(blockIdx.x, ntile, tm, tn);
    const int m0 = tm * kWT, n0 = tn * kWT;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;  // 16 x 16 threads, 4 x 4 pairs each
    int id[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) id[u][v] = 0;
    if (threadIdx.x < kWT) {
        cntA[threadIdx.x] = 0;
        cntB[threadIdx.x] = 0;
    }
    const int Lw = (L + 3) / 4;
    for (int w0 = 0; w0 < Lw; w0 += kWChunk) {
        const int nw = min(kWChunk, Lw - w0);
        __syncthreads();
        // Stage words; bytes beyond L are 0xff in A and 0xfe in B so they never match.
        for (int k = threadIdx.x; k < kWT * kWChunk; k += blockDim.x) {
            const int r = k / kWChunk, c = k % kWChunk;
            uint32_t va = 0xffffffffu, vb = 0xfefefefeu;
            if (c < nw) {
                const int wi = w0 + c;
                const int ma = m0 + r, nb = n0 + r;
                uint32_t xa = 0, xb = 0;
#pragma unroll
                for (int k4 = 0; k4 < 4; ++k4) {
                    const int site = wi * 4 + k4;
                    const uint32_t ca = (ma < N && site < L) ? X[(size_t)ma * L + site] : 0xffu;
                    const uint32_t cb = (nb < N && site < L) ? X[(size_t)nb * L + site] : 0xfeu;
                    xa |= ca << (8 * k4);
                    xb |= cb << (8 * k4);
                }
                va = xa;
                vb = xb;
            }
            A[r][c] = va;
            B[r][c] = vb;
        }
        __syncthreads();
        uint32_t acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = 0;
        for (int c = 0; c < nw; ++c) {
            uint32_t ra[4], rb[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) ra[u] = A[ty + 16 * u][c];
#pragma unroll
            for (int v = 0; v < 4; ++v) rb[v] = B[tx + 16 * v][c];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] += match_bytes(ra[u], rb[v]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) id[u][v] += fold_bytes(acc[u][v]);
    }
    // Credit qualifying pairs.
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int rm = ty + 16 * u, rn = tx + 16 * v;
            const int m = m0 + rm, n = n0 + rn;
            if (m >= N || n >= N || id[u][v] < thr) continue;
            if (tm == tn) {
                if (rm < rn) {
                    atomicAdd(&cntA[rm], 1);
                    atomicAdd(&cntB[rn], 1);
                } else if (rm == rn) {
                    atomicAdd(&cntA[rm], 1);  // self-identity, counted once
                }
            } else {
                atomicAdd(&cntA[rm], 1);
                atomicAdd(&cntB[rn], 1);
            }
        }
    __syncthreads();
    if (threadIdx.x < kWT) {
        const int m = m0 + threadIdx.x, n = n0 + threadIdx.x;
        if (m < N && cntA[threadIdx.x]) atomicAdd(&cnt[m], cntA[threadIdx.x]);
        if (n < N && cntB[threadIdx.x]) atomicAdd(&cnt[n], cntB[threadIdx.x]);
    }
}

// ----------------------------------------------------------------------------
// Bit-sliced identity counts (the same counts as k_identity).  A pre-pass
// stores every sequence as 8 bit planes of its symbol bytes, 32 positions
// per word (word w of a sequence = 8 consecutive uint32, plane p holding
// bit p of the symbols at positions 32w .. 32w+31; zero beyond L), and ORs
// all symbols into one flag word.  For a pair, OR over the planes of
// (a_p XOR b_p) marks the positions whose symbols differ, so a word of 32
// positions costs one logic op per plane and a popcount: identity = L -
// mismatches.  Planes above the highest bit any symbol uses are all zero
// and skipped (5 planes for alphabets up to 32 symbols).
// ----------------------------------------------------------------------------
constexpr int kBP = 8;        // bit planes stored (symbol bytes)
constexpr int kBWChunk = 8;   // words (of 32 positions) per staged chunk

// One warp per (sequence, word): lane k holds position 32w + k.
__global__ void __launch_bounds__(256) k_bitslice(const uint8_t *__restrict__ X, int N, int L, int Lw,
                                                  uint32_t *__restrict__ planes, unsigned *__restrict__ used)
{
    const long long warp_id = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp_id >= (long long)N * Lw) return;  // whole warps leave together
    const int n = (int)(warp_id / Lw), wd = (int)(warp_id % Lw);
    const int pos = wd * 32 + lane;
    const uint32_t b = pos < L ? X[(size_t)n * L + pos] : 0u;
    uint32_t mine = 0, any = 0;
#pragma unroll
    for (int pl = 0; pl < kBP; ++pl) {
        const uint32_t word = __ballot_sync(0xffffffffu, (b >> pl) & 1u);
        if (lane == pl) mine = word;
        any |= word ? (1u << pl) : 0u;
    }
    if (lane < kBP) planes[((size_t)n * Lw + wd) * kBP + lane] = mine;
    if (lane == 0 && any) atomicOr(used, any);
}

// 4 x 4 pairs of one thread over one word: mismatches from the first NP planes.
template <int NP>
__device__ __forceinline__ void pair_words(const uint4 (&a)[4][2], const uint4 (&b)[4][2], int (&mism)[4][4])
{
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const uint32_t pa[8] = {a[u][0].x, a[u][0].y, a[u][0].z, a[u][0].w,
                                    a[u][1].x, a[u][1].y, a[u][1].z, a[u][1].w};
            const uint32_t pb[8] = {b[v][0].x, b[v][0].y, b[v][0].z, b[v][0].w,
                                    b[v][1].x, b[v][1].y, b[v][1].z, b[v][1].w};
            uint32_t d = pa[0] ^ pb[0];
#pragma unroll
            for (int pl = 1; pl < NP; ++pl) d |= pa[pl] ^ pb[pl];
            mism[u][v] += __popc(d);
        }
}

// Position in the row-major enumeration of the upper triangle of tile pairs,
// advanced by a fixed stride without re-walking the rows.
struct TriCursor {
    int r, rem;  // tile pair (r, r + rem)
    __device__ __forceinline__ void init(long long t, int nt)
    {
        r = 0;
        long long x = t;
        while (r < nt && x >= nt - r) {
            x -= nt - r;
            ++r;
        }
        rem = (int)x;
    }
    __device__ __forceinline__ void advance(int by, int nt)
    {
        long long x = (long long)rem + by;
        while (r < nt && x >= nt - r) {
            x -= nt - r;
            ++r;
        }
        rem = (int)x;
    }
};

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, bool valid)
{
    // src-size 0 fills the 16 bytes with zeros (rows past N, words past Lw)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}

constexpr int kIdRow4 = 2 * kBWChunk + 1;  // uint4 per staged sequence (odd: conflict-free 128-bit reads)
constexpr int kIdBlocksPerSM = 2;          // latency is hidden by the double buffer, not by occupancy
constexpr size_t kIdSmem = (size_t)2 * 2 * kWT * kIdRow4 * sizeof(uint4) + 2 * kWT * sizeof(int);

// The 4 x 4 pairs of one thread over nw staged words; only the planes in
// use are loaded (five: planes 0-3 as one 16-byte word and plane 4 as 4
// bytes, which cuts the shared-memory wavefronts of the loads).
template <int NP>
__device__ __forceinline__ void compare_chunk(const uint4 *__restrict__ A, const uint4 *__restrict__ B, int nw,
                                              int ty, int tx, int (&mism)[4][4])
{
    for (int c = 0; c < nw; ++c) {
        uint4 ra[4][2], rb[4][2];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint4 *pa = A + (ty + 16 * u) * kIdRow4 + 2 * c;
            ra[u][0] = pa[0];
            if (NP > 4) {
                if (NP > 5) ra[u][1] = pa[1];
                else ra[u][1].x = reinterpret_cast<const uint32_t *>(pa + 1)[0];
            }
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const uint4 *pb = B + (tx + 16 * v) * kIdRow4 + 2 * c;
            rb[v][0] = pb[0];
            if (NP > 4) {
                if (NP > 5) rb[v][1] = pb[1];
                else rb[v][1].x = reinterpret_cast<const uint32_t *>(pb + 1)[0];
            }
        }
        pair_words<NP>(ra, rb, mism);
    }
}

// Persistent over tile pairs (64 x 64 sequences) and their 256-position
// chunks: the next step's planes are copied into the other half of a
// double buffer (cp.async) while this step's pairs are compared, so the
// loads of a tile pair overlap the comparisons of the previous one.
__global__ void __launch_bounds__(256, kIdBlocksPerSM) k_identity_bs(const uint32_t *__restrict__ planes,
                                                                     const unsigned *__restrict__ used, int N, int L,
                                                                     int Lw, int thr, int ntile, long long npairs,
                                                                     int *__restrict__ cnt)
{
    extern __shared__ __align__(16) unsigned char id_smem[];
    uint4 *buf = reinterpret_cast<uint4 *>(id_smem);  // [2 halves][A, B][kWT][kIdRow4]
    int *cntA = reinterpret_cast<int *>(buf + 2 * 2 * kWT * kIdRow4);
    int *cntB = cntA + kWT;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;  // 16 x 16 threads, 4 x 4 pairs each
    const bool five = (*used >> 5) == 0u;                    // every symbol < 32
    const uint4 *P4 = reinterpret_cast<const uint4 *>(planes);
    const int nch = (Lw + kBWChunk - 1) / kBWChunk;
    const long long mine = blockIdx.x < npairs ? (npairs - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const long long steps = mine * nch;
    if (threadIdx.x < kWT) {
        cntA[threadIdx.x] = 0;
        cntB[threadIdx.x] = 0;
    }
    TriCursor cc, pc;  // tile pair being compared / being fetched
    cc.init(blockIdx.x, ntile);
    pc = cc;
    int cch = 0, pch = 0;  // their chunks
    auto fetch = [&](int half) {
        const int m0 = pc.r * kWT, n0 = (pc.r + pc.rem) * kWT, w0 = pch * kBWChunk;
        const int nw = min(kBWChunk, Lw - w0);
        uint4 *A = buf + (size_t)half * 2 * kWT * kIdRow4, *B = A + kWT * kIdRow4;
        for (int k = threadIdx.x; k < kWT * 2 * kBWChunk; k += blockDim.x) {
            const int r = k / (2 * kBWChunk), c2 = k % (2 * kBWChunk);
            const int ma = m0 + r, nb = n0 + r;
            const bool in = (c2 >> 1) < nw;
            const bool va = in && ma < N, vb = in && nb < N;
            cp_async16((uint32_t)__cvta_generic_to_shared(A + r * kIdRow4 + c2),
                       va ? P4 + ((size_t)ma * Lw + w0) * 2 + c2 : P4, va);
            cp_async16((uint32_t)__cvta_generic_to_shared(B + r * kIdRow4 + c2),
                       vb ? P4 + ((size_t)nb * Lw + w0) * 2 + c2 : P4, vb);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        if (++pch == nch) {
            pch = 0;
            pc.advance(gridDim.x, ntile);
        }
    };
    int mism[4][4];
    if (steps > 0) fetch(0);
    for (long long s = 0; s < steps; ++s) {
        if (s + 1 < steps) {
            fetch((int)((s + 1) & 1));
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();
        if (cch == 0) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) mism[u][v] = 0;
        }
        const uint4 *A = buf + (size_t)(s & 1) * 2 * kWT * kIdRow4, *B = A + kWT * kIdRow4;
        const int nw = min(kBWChunk, Lw - cch * kBWChunk);
        if (five)
            compare_chunk<5>(A, B, nw, ty, tx, mism);
        else
            compare_chunk<8>(A, B, nw, ty, tx, mism);
        if (cch == nch - 1) {
            // Credit qualifying pairs (identity = L - mismatches >= thr).
            const int tm = cc.r, tn = cc.r + cc.rem, m0 = tm * kWT, n0 = tn * kWT;
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const int rm = ty + 16 * u, rn = tx + 16 * v;
                    const int m = m0 + rm, n = n0 + rn;
                    if (m >= N || n >= N || L - mism[u][v] < thr) continue;
                    if (tm == tn) {
                        if (rm < rn) {
                            atomicAdd(&cntA[rm], 1);
                            atomicAdd(&cntB[rn], 1);
                        } else if (rm == rn) {
                            atomicAdd(&cntA[rm], 1);  // self-identity, counted once
                        }
                    } else {
                        atomicAdd(&cntA[rm], 1);
                        atomicAdd(&cntB[rn], 1);
                    }
                }
            __syncthreads();
            if (threadIdx.x < kWT) {
                const int m = m0 + threadIdx.x, n = n0 + threadIdx.x;
                if (m < N && cntA[threadIdx.x]) atomicAdd(&cnt[m], cntA[threadIdx.x]);
                if (n < N && cntB[threadIdx.x]) atomicAdd(&cnt[n], cntB[threadIdx.x]);
                cntA[threadIdx.x] = 0;
                cntB[threadIdx.x] = 0;
            }
        }
        __syncthreads();  // this half is refilled by the fetch two steps on
        if (++cch == nch) {
            cch = 0;
            cc.advance(gridDim.x, ntile);
        }
    }
}

__global__ void k_weights_finalize(const int *__restrict__ cnt, int N, float *__restrict__ w,
                                   double *meff)
{
    __shared__ double red[1024];
    double s = 0.0;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const double v = 1.0 / (double)cnt[k];
        w[k] = (float)v;
        s += v;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *meff = red[0];
}

int chain_tile(int q)
{
    // Largest power-of-two tile whose int32 histograms fit in ~120 KB.
    int ts = 32;
    while (ts > 1 && (size_t)ts * ts * q * q * 4 > 120 * 1024) ts >>= 1;
    return ts;
}

int data_tile(int q)
{
    int ts = 32;
    while (ts > 1 && (size_t)ts * ts * q * q * 8 > 120 * 1024) ts >>= 1;
    return ts;
}

template <int TS>
int launch_chain_pairs(const uint8_t *s, int M, int L, int q, int32_t *counts, cudaStream_t st)
{
    const int nt = (L + TS - 1) / TS;
    const int npairs = nt * (nt + 1) / 2;
    const size_t smem = (size_t)TS * TS * q * q * 4 + (size_t)kChunk * 2 * TS;
    auto kern = k_chain_pairs<TS>;
    BM_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<npairs, 512, smem, st>>>(s, M, L, q, nt, counts);
    BM_CK_LAUNCH("k_chain_pairs");
    return BM_OK;
}

template <int TS>
int launch_data_pairs(const uint8_t *X, const float *w, int N, int L, int q, double meff,
                      double alpha, float *fi, float *fij, cudaStream_t st)
{
    const int nt = (L + TS - 1) / TS;
    const int npairs = nt * (nt + 1) / 2;
    const size_t smem = (size_t)TS * TS * q * q * 8 + (size_t)kChunk * 8 + (size_t)kChunk * 2 * TS;
    auto kern = k_data_pairs<TS>;
    BM_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<npairs, 512, smem, st>>>(X, w, N, L, q, nt, meff, alpha, fi, fij);
    BM_CK_LAUNCH("k_data_pairs");
    return BM_OK;
}

}  // namespace

int bm_launch_chain_stats(const uint8_t *s, int M, int L, int q, int32_t *counts, cudaStream_t st)
{
    switch (chain_tile(q)) {
    case 32: return launch_chain_pairs<32>(s, M, L, q, counts, st);
    case 16: return launch_chain_pairs<16>(s, M, L, q, counts, st);
    case 8: return launch_chain_pairs<8>(s, M, L, q, counts, st);
    case 4: return launch_chain_pairs<4>(s, M, L, q, counts, st);
    case 2: return launch_chain_pairs<2>(s, M, L, q, counts, st);
    default: return launch_chain_pairs<1>(s, M, L, q, counts, st);
    }
}

int bm_launch_data_stats(const uint8_t *msa, const float *w, int N, int L, int q, double alpha,
                         int /*frac_bits*/, double meff, float *fi, float *fij,
                         unsigned long long * /*acc_fi*/, cudaStream_t st)
{
    switch (data_tile(q)) {
    case 32: return launch_data_pairs<32>(msa, w, N, L, q, meff, alpha, fi, fij, st);
    case 16: return launch_data_pairs<16>(msa, w, N, L, q, meff, alpha, fi, fij, st);
    case 8: return launch_data_pairs<8>(msa, w, N, L, q, meff, alpha, fi, fij, st);
    case 4: return launch_data_pairs<4>(msa, w, N, L, q, meff, alpha, fi, fij, st);
    case 2: return launch_data_pairs<2>(msa, w, N, L, q, meff, alpha, fi, fij, st);
    default: return launch_data_pairs<1>(msa, w, N, L, q, meff, alpha, fi, fij, st);
    }
}

int bm_launch_weight_sum(const float *w, int N, double *out3, cudaStream_t st)
{
    k_weight_sum<<<1, 1024, 0, st>>>(w, N, out3);
    BM_CK_LAUNCH("k_weight_sum");
    return BM_OK;
}

size_t bm_seq_weights_planes_bytes(int N, int L)
{
    return (size_t)N * kBP * ((L + 31) / 32) * sizeof(uint32_t) + 16;  // + the used-bits word
}

int bm_launch_seq_weights_bs(const uint8_t *msa, int N, int L, int thr, float *w, int *cnt, uint32_t *planes,
                             double *meff_dev, cudaStream_t st)
{
    const int Lw = (L + 31) / 32;
    unsigned *used = reinterpret_cast<unsigned *>(planes + (size_t)N * kBP * Lw);
    BM_CK(cudaMemsetAsync(cnt, 0, (size_t)N * sizeof(int), st));
    BM_CK(cudaMemsetAsync(used, 0, sizeof(unsigned), st));
    const long long warps = (long long)N * Lw;
    k_bitslice<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(msa, N, L, Lw, planes, used);
    BM_CK_LAUNCH("k_bitslice");
    const int ntile = (N + kWT - 1) / kWT;
    const long long npairs = (long long)ntile * (ntile + 1) / 2;
    int dev = 0, nsm = 0;
    BM_CK(cudaGetDevice(&dev));
    BM_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    BM_CK(cudaFuncSetAttribute(k_identity_bs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kIdSmem));
    const int grid = (int)std::max<long long>(1, std::min<long long>(npairs, (long long)nsm * kIdBlocksPerSM));
    k_identity_bs<<<grid, 256, kIdSmem, st>>>(planes, used, N, L, Lw, thr, ntile, npairs, cnt);
    BM_CK_LAUNCH("k_identity_bs");
    k_weights_finalize<<<1, 1024, 0, st>>>(cnt, N, w, meff_dev);
    BM_CK_LAUNCH("k_weights_finalize");
    return BM_OK;
}

int bm_launch_seq_weights(const uint8_t *msa, int N, int L, int thr, float *w, int *cnt,
                          double *meff_dev, cudaStream_t st)
{
    BM_CK(cudaMemsetAsync(cnt, 0, (size_t)N * sizeof(int), st));
    const int ntile = (N + kWT - 1) / kWT;
    const long long npairs = (long long)ntile * (ntile + 1) / 2;
    if (npairs > 0x7fffffffLL) return bm_fail(BM_EINVAL, "bm_seq_weights: N too large");
    k_identity<<<(unsigned)npairs, 256, 0, st>>>(msa, N, L, thr, ntile, cnt);
    BM_CK_LAUNCH("k_identity");
    k_weights_finalize<<<1, 1024, 0, st>>>(cnt, N, w, meff_dev);
    BM_CK_LAUNCH("k_weights_finalize");
    return BM_OK;
}
