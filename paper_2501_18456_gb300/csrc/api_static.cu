// bm_seq_weights_static: the sequence-weight computation of bm_seq_weights
// without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need
// the weights: code running while another framework's caching allocator has
// reserved the device's memory, latency-critical serving loops that must
// not enter the driver's allocator (cudaMalloc / cudaFree can synchronise
// the device), and embedders that hand this library a fixed memory budget.
// For them the identity counters and the M_eff accumulator live in one
// file-scope device array of fixed size, reserved when the library is
// loaded and held on every GPU that loads it until the process exits.
//
// Host code cannot use the array's name as a device address (in host code
// it names a host-side stand-in), so the first call on each device, with
// that device current, looks the address up with cudaGetSymbolAddress and
// caches it.  That first call should therefore happen before any stream
// capture begins.  The cached address lives as long as the process; a
// cudaDeviceReset unloads the module and with it the array, so the entry
// point must not be used on that device again afterwards.  All calls share the one array: calls whose work overlaps
// on the GPU (different streams, or different host threads) race on it.
// The counters are cleared at the start of every call.
#include "bm_internal.cuh"

#include <math.h>

#include <mutex>

namespace {

constexpr int kStaticMaxN = BM_SEQ_WEIGHTS_STATIC_MAX_N;
constexpr size_t kHeaderBytes = 256;  // M_eff (double) at offset 0, counters after

static __device__ __align__(256) unsigned char g_seqw_scratch[kHeaderBytes + (size_t)kStaticMaxN * sizeof(int)];

constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

int scratch_for_current_device(void **out)
{
    int dev = 0;
    BM_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices)
        return bm_fail(BM_EINVAL, "bm_seq_weights_static: device ordinal %d unsupported", dev);
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_seqw_scratch);
        if (e != cudaSuccess) return bm_cuda_fail(e, "cudaGetSymbolAddress(g_seqw_scratch)");
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return BM_OK;
}

}  // namespace

extern "C" int bm_seq_weights_static(const uint8_t *msa_dev, int N, int L, double seqid,
                                     float *w_dev, double *meff_host, void *stream)
{
    if (!msa_dev || !w_dev) return bm_fail(BM_EINVAL, "bm_seq_weights_static: NULL argument");
    if (N < 1 || L < 1 || L > 4096)
        return bm_fail(BM_EINVAL, "bm_seq_weights_static: bad N=%d or L=%d", N, L);
    if (N > kStaticMaxN)
        return bm_fail(BM_EINVAL,
                       "bm_seq_weights_static: N=%d exceeds the static scratch limit of %d sequences",
                       N, kStaticMaxN);
    if (!(seqid > 0.0 && seqid <= 1.0))
        return bm_fail(BM_EINVAL, "bm_seq_weights_static: seqid out of (0,1]");
    void *base = nullptr;
    int rc = scratch_for_current_device(&base);
    if (rc != BM_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    double *meff_dev = (double *)base;
    int *cnt = (int *)((unsigned char *)base + kHeaderBytes);
    const int thr = (int)ceil(seqid * L - 1e-9);
    rc = bm_launch_seq_weights(msa_dev, N, L, thr, w_dev, cnt, meff_dev, st);
    if (rc != BM_OK || !meff_host) return rc;
    double meff = 0.0;
    BM_CK(cudaMemcpyAsync(&meff, meff_dev, sizeof(double), cudaMemcpyDeviceToHost, st));
    BM_CK(cudaStreamSynchronize(st));
    *meff_host = meff;
    return BM_OK;
}
