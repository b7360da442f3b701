// Error plumbing and the device exclusive scan used by setup (coarse
// numbering, row pointers of R, A_c and scratch buffers).
#include <cstdio>
#include <mutex>

#include "common.cuh"

namespace pr {

std::atomic<long long> g_launches{0};
thread_local long long g_thread_launches = 0;

void fail(pair_status st, const std::string &msg) { throw Error{st, msg}; }

// free device memory as the library can use it: what the device reports free plus
// what its pool holds mapped but unused
size_t available_device_bytes() {
    size_t freeb = 0, totb = 0;
    cuda_check(cudaMemGetInfo(&freeb, &totb), "cudaMemGetInfo", __FILE__, __LINE__);
    cudaMemPool_t pool = device_pool();
    unsigned long long reserved = 0, used = 0;
    cuda_check(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved),
               "cudaMemPoolGetAttribute", __FILE__, __LINE__);
    cuda_check(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used), "cudaMemPoolGetAttribute",
               __FILE__, __LINE__);
    return freeb + (size_t)(reserved > used ? reserved - used : 0);
}

cudaMemPool_t device_pool() {
    static std::mutex mu;
    static cudaMemPool_t pools[256] = {};
    int dev = 0;
    cuda_check(cudaGetDevice(&dev), "cudaGetDevice", __FILE__, __LINE__);
    if (dev < 0 || dev >= 256) fail(PAIR_ERR_UNSUPPORTED, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        cuda_check(cudaMemPoolCreate(&pool, &props), "cudaMemPoolCreate", __FILE__, __LINE__);
        unsigned long long keep = ~0ULL;
        cuda_check(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep),
                   "cudaMemPoolSetAttribute", __FILE__, __LINE__);
        pools[dev] = pool;
    }
    return pools[dev];
}

void cuda_check(cudaError_t e, const char *what, const char *file, int line) {
    if (e == cudaSuccess) return;
    cudaGetLastError();
    char buf[512];
    snprintf(buf, sizeof buf, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    pair_status st = (e == cudaErrorMemoryAllocation) ? PAIR_ERR_OOM : PAIR_ERR_CUDA;
    fail(st, buf);
}

namespace {
constexpr int SCAN_BS = 256;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_BS * SCAN_ITEMS;

__device__ long long block_excl_scan(long long v, long long *sh, long long *total) {
    // Hillis-Steele over the block in shared memory (SCAN_BS threads)
    int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int off = 1; off < SCAN_BS; off <<= 1) {
        long long add = t >= off ? sh[t - off] : 0;
        __syncthreads();
        sh[t] += add;
        __syncthreads();
    }
    long long incl = sh[t];
    *total = sh[SCAN_BS - 1];
    __syncthreads();
    return incl - v;
}

template <class In>
__global__ void k_tile_sums(const In *in, int n, long long *sums) {
    __shared__ long long sh[SCAN_BS];
    long long base = (long long)blockIdx.x * SCAN_TILE;
    long long s = 0;
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        long long i = base + (long long)threadIdx.x * SCAN_ITEMS + k;
        if (i < n) s += in[i];
    }
    long long tot;
    block_excl_scan(s, sh, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_scan_sums(long long *sums, int nb) {
    // one block: exclusive scan of the tile sums in chunks, carrying the total
    __shared__ long long sh[SCAN_BS];
    long long carry = 0;
    for (int c0 = 0; c0 < nb; c0 += SCAN_BS) {
        int i = c0 + threadIdx.x;
        long long v = i < nb ? sums[i] : 0;
        long long tot;
        long long ex = block_excl_scan(v, sh, &tot);
        if (i < nb) sums[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) sums[nb] = carry;
}

// (in may be out: each thread reads its items before writing them)
template <class In, class Out>
__global__ void k_scan_tiles(const In *in, int n, const long long *sums, Out *out, long long *total_out,
                             int nb) {
    __shared__ long long sh[SCAN_BS];
    long long base = (long long)blockIdx.x * SCAN_TILE;
    long long v[SCAN_ITEMS];
    long long s = 0;
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        long long i = base + (long long)threadIdx.x * SCAN_ITEMS + k;
        v[k] = i < n ? in[i] : 0;
        s += v[k];
    }
    long long tot;
    long long ex = block_excl_scan(s, sh, &tot) + sums[blockIdx.x];
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        long long i = base + (long long)threadIdx.x * SCAN_ITEMS + k;
        if (i < n) out[i] = (Out)ex;
        ex += v[k];
    }
    if (blockIdx.x == nb - 1 && threadIdx.x == 0) {
        out[n] = (Out)sums[nb];
        *total_out = sums[nb];
    }
}
}  // namespace

long long scan_exclusive(const int *in, int *out, int n, cudaStream_t s, bool want_total) {
    if (n <= 0) {
        PR_CUDA(cudaMemsetAsync(out, 0, sizeof(int), s));
        return 0;
    }
    int nb = (int)blocks_for(n, SCAN_TILE);
    long long *sums = dmalloc<long long>(nb + 2, s);
    k_tile_sums<int><<<nb, SCAN_BS, 0, s>>>(in, n, sums);
    PR_LAUNCH();
    k_scan_sums<<<1, SCAN_BS, 0, s>>>(sums, nb);
    PR_LAUNCH();
    k_scan_tiles<int, int><<<nb, SCAN_BS, 0, s>>>(in, n, sums, out, sums + nb + 1, nb);
    PR_LAUNCH();
    long long total = 0;
    if (want_total) {
        PR_CUDA(cudaMemcpyAsync(&total, sums + nb + 1, sizeof(long long), cudaMemcpyDeviceToHost, s));
        PR_CUDA(cudaStreamSynchronize(s));
        if (total > 0x7fffffffLL)
            fail(PAIR_ERR_UNSUPPORTED, "scan total exceeds int32: batch too large for 32-bit indices");
    }
    dfree(sums, s);
    return total;
}

long long scan_exclusive_ll(long long *v, int n, cudaStream_t s) {
    if (n <= 0) {
        PR_CUDA(cudaMemsetAsync(v, 0, sizeof(long long), s));
        return 0;
    }
    int nb = (int)blocks_for(n, SCAN_TILE);
    long long *sums = dmalloc<long long>(nb + 2, s);
    k_tile_sums<long long><<<nb, SCAN_BS, 0, s>>>(v, n, sums);
    PR_LAUNCH();
    k_scan_sums<<<1, SCAN_BS, 0, s>>>(sums, nb);
    PR_LAUNCH();
    k_scan_tiles<long long, long long><<<nb, SCAN_BS, 0, s>>>(v, n, sums, v, sums + nb + 1, nb);
    PR_LAUNCH();
    long long total = 0;
    PR_CUDA(cudaMemcpyAsync(&total, sums + nb + 1, sizeof(long long), cudaMemcpyDeviceToHost, s));
    PR_CUDA(cudaStreamSynchronize(s));
    dfree(sums, s);
    return total;
}

}  // namespace pr
