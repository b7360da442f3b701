// Residual and residual norm with no device allocation.
//
// Some callers cannot allocate device memory at the point where they need a
// residual: code running under a memory pool or arena that forbids
// cudaMalloc/cudaFree (allocation would synchronise the device or escape the
// arena's accounting), or a host that has reserved all device memory for its
// own buffers.  This variant of the level-0 residual kernel keeps its only
// scratch (one partial sum of squares per thread block) in a file-scope static
// device array, so the call allocates nothing; the caller still passes A, b, x
// and the outputs.
//
// The array's name is a host-side stand-in in host code, so the host obtains
// its device address with cudaGetSymbolAddress once per device (the first
// call on a device does this; make that first call before any stream capture)
// and passes the address to the kernels.  The address is cached with the id of
// the CUDA context it belongs to: after a device reset (a new primary context,
// the module loaded again) the next call looks the address up afresh instead
// of using the old one.  Every call shares the array: calls
// whose kernels overlap on the GPU race on it.  Each call writes every partial
// it later reads, so nothing has to be cleared between calls.
#include <cuda.h>   // CUcontext / CUresult types only; the functions come from the runtime

#include <mutex>

#include "common.cuh"

namespace {

constexpr int NA_BS = 256;
constexpr int NA_MAX_BLOCKS = PAIR_NOALLOC_MAX_ROWS / NA_BS;

__device__ __align__(256) double g_noalloc_partials[NA_MAX_BLOCKS];

__global__ void k_na_residual(int n, const int *rowptr, const int *col, const double *val, const double *b,
                              const double *x, double *r, double *partials) {
    __shared__ double sh[NA_BS / 32];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double s2 = 0.0;
    if (i < n) {
        double acc = 0.0;
        for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) acc += val[p] * x[col[p]];
        acc = b[i] - acc;
        r[i] = acc;
        s2 = acc * acc;
    }
    for (int o = 16; o > 0; o >>= 1) s2 += __shfl_down_sync(0xffffffffu, s2, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < NA_BS / 32; ++k) t += sh[k];
        partials[blockIdx.x] = t;
    }
}

// fixed-order sum of the block partials (deterministic)
__global__ void k_na_norm(int nb, const double *partials, double *out) {
    __shared__ double sh[NA_BS];
    double t = 0.0;
    for (int k = threadIdx.x; k < nb; k += NA_BS) t += partials[k];
    sh[threadIdx.x] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < NA_BS; ++k) s += sh[k];
        out[0] = sqrt(s);
    }
}

std::mutex g_na_mutex;
double *g_na_addr[256] = {nullptr};
unsigned long long g_na_ctx[256] = {0};

// id of the calling thread's current CUDA context (0 if none yet); the driver
// functions are obtained through the runtime, so libpair does not link libcuda
unsigned long long current_context_id() {
    typedef CUresult (*get_current_fn)(CUcontext *);
    typedef CUresult (*get_id_fn)(CUcontext, unsigned long long *);
    static get_current_fn get_current = nullptr;
    static get_id_fn get_id = nullptr;
    if (!get_current || !get_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        PR_CUDA(cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1));
        PR_CUDA(cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2));
        PR_REQUIRE(f1 && f2 && q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess,
                   PAIR_ERR_CUDA, "driver context queries unavailable");
        get_current = reinterpret_cast<get_current_fn>(f1);
        get_id = reinterpret_cast<get_id_fn>(f2);
    }
    CUcontext c = nullptr;
    if (get_current(&c) != CUDA_SUCCESS || !c) return 0;
    unsigned long long id = 0;
    return get_id(c, &id) == CUDA_SUCCESS ? id : 0;
}

double *scratch_address() {
    int dev = 0;
    PR_CUDA(cudaGetDevice(&dev));
    PR_REQUIRE(dev >= 0 && dev < 256, PAIR_ERR_UNSUPPORTED, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_na_mutex);
    unsigned long long ctx = current_context_id();
    if (!g_na_addr[dev] || ctx == 0 || ctx != g_na_ctx[dev]) {
        void *p = nullptr;   // this call also makes the device's primary context current
        PR_CUDA(cudaGetSymbolAddress(&p, g_noalloc_partials));
        g_na_addr[dev] = static_cast<double *>(p);
        g_na_ctx[dev] = current_context_id();
    }
    return g_na_addr[dev];
}

}  // namespace

extern "C" pair_status pair_residual_norm_noalloc(const pair_csr *A, const double *b, const double *x, double *r,
                                                  double *rnorm, void *stream) {
    try {
        PR_REQUIRE(A && b && x && r && rnorm && A->rowptr, PAIR_ERR_ARG, "pair_residual_norm_noalloc: null argument");
        PR_REQUIRE(A->n >= 1 && A->nnz >= 0 && (A->nnz == 0 || (A->col && A->val)), PAIR_ERR_ARG,
                   "pair_residual_norm_noalloc: empty or malformed matrix");
        PR_REQUIRE(A->n <= PAIR_NOALLOC_MAX_ROWS, PAIR_ERR_UNSUPPORTED,
                   "pair_residual_norm_noalloc: n = " + std::to_string(A->n) + " exceeds the static scratch limit of " +
                       std::to_string(PAIR_NOALLOC_MAX_ROWS) + " rows");
        double *partials = scratch_address();
        pr::set_last_error("");
        cudaStream_t s = (cudaStream_t)stream;
        int nb = (int)pr::blocks_for(A->n, NA_BS);
        k_na_residual<<<nb, NA_BS, 0, s>>>(A->n, A->rowptr, A->col, A->val, b, x, r, partials);
        PR_LAUNCH();
        k_na_norm<<<1, NA_BS, 0, s>>>(nb, partials, rnorm);
        PR_LAUNCH();
        return PAIR_OK;
    } catch (const pr::Error &e) {
        pr::set_last_error(e.msg);
        return e.st;
    } catch (...) {
        pr::set_last_error("pair_residual_norm_noalloc: internal error");
        return PAIR_ERR_CUDA;
    }
}
