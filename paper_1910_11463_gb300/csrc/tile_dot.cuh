// Row dot products of a CSR-like store, staged through shared memory by TMA bulk
// copies: the work of the coarse-level Jacobi sweeps (Sec. 1.2 relaxation, on the
// CF-split rows) and of the restriction b_c = R b = Z b_F + b_C (Sec. 1.2, ℓAIR).
//
// A persistent grid of 256-thread CTAs walks the rows in tiles of 256/G rows (G
// lanes per row).  For each tile, one thread issues two cp.async.bulk copies
// (columns and values of the tile's entries, widened to 16-byte boundaries) that
// complete on an mbarrier; two stages are in flight, so the next tile streams from
// HBM while the current one is computed.  The lanes then read entries from shared
// memory and gather the vector (L2-resident) per entry.  Per lane the terms are
// added in ascending entry order (lane g takes entries g, g+G, ...), then a fixed
// shuffle tree, the same order as a G-lane row loop.
//
// A tile whose window is empty, larger than the stage, or ends past the store's
// last entry (the widened window must stay inside the arrays) is computed from
// global memory instead.  Every wait on an mbarrier gives up after about one
// second of global time: the CTA then sets DERR_TIMEOUT in the error word, waits
// (again bounded) for its own copies in flight and returns.
#pragma once

#include "common.cuh"

namespace pr {
namespace tile {

constexpr int BS = 256;
constexpr int CTAS_PER_SM = 6;

template <class T>
struct Job {
    int k0, k1;              // rows [k0, k1) of the store
    long long nnz;           // entries in col/val (copies never read past them)
    const int *ptr, *col;    // row offsets (row k: [ptr[k], ptr[k+1])), columns
    const T *val;
    const T *in;             // gathered vector
    const int *srow;         // sweeps: row index of store row k
    const T *dinv, *b;
    T *out;
    double *x64;             // F sweep: optional fold target; final C sweep: target
    const int *cpts;         // restriction: fine row of coarse point k
    const int *active, *rowdir;
    int *err;
};

enum Mode : int { F_SWEEP = 0, C_SWEEP = 1, C_SWEEP_FINAL = 2, RESTRICT = 3 };

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// true once the phase with this parity has completed; false after ~1 s
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity) {
    if (mbar_test(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (mbar_test(bar, parity)) return true;
        if (global_ns() - t0 > 1000000000ull) return false;
    }
}

template <class T, int G, int MODE>
__global__ void __launch_bounds__(BS) k_tile_dot(Job<T> j, int ntiles) {
    constexpr int TR = BS / G;                               // rows per tile
    constexpr int ECAP = sizeof(T) == 8 ? 1536 : 2048;       // entries per stage
    __shared__ __align__(128) int s_col[2][ECAP];
    __shared__ __align__(128) T s_val[2][ECAP];
    __shared__ __align__(8) unsigned long long bar[2];

    const int g = threadIdx.x % G, lr = threadIdx.x / G;
    if (threadIdx.x == 0) {
        mbar_init(&bar[0]);
        mbar_init(&bar[1]);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();

    // entry window of tile t, widened to multiples of 4 entries (16 bytes of
    // columns); cnt = 0: compute the tile from global memory
    auto window = [&](int t, int &a0, int &cnt) {
        const int rs = j.k0 + t * TR, re = min(rs + TR, j.k1);
        const int e0 = j.ptr[rs], e1 = j.ptr[re];
        a0 = e0 & ~3;
        const long long a1 = ((long long)e1 + 3) & ~3LL;
        cnt = (int)(a1 - a0);
        if (cnt <= 0 || cnt > ECAP || a1 > j.nnz) cnt = 0;
    };
    unsigned pending = 0;   // thread 0: stages with a copy in flight
    auto issue = [&](int t, int s) {
        if (t >= ntiles) return;
        int a0, cnt;
        window(t, a0, cnt);
        if (cnt == 0) return;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&bar[s], (unsigned)(cnt * (4 + (int)sizeof(T))));
        bulk_load(s_col[s], j.col + a0, (unsigned)cnt * 4u, &bar[s]);
        bulk_load(s_val[s], j.val + a0, (unsigned)cnt * (unsigned)sizeof(T), &bar[s]);
        pending |= 1u << s;
    };
    if (threadIdx.x == 0) {
        issue(blockIdx.x, 0);
        issue(blockIdx.x + gridDim.x, 1);
    }

    unsigned phase = 0;   // bit s: parity of the next completion on stage s
    int it = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
        const int s = it & 1;
        const int rs = j.k0 + t * TR, re = min(rs + TR, j.k1);
        int a0, cnt;
        window(t, a0, cnt);
        const int k = rs + lr;
        const bool valid = k < re;
        int p0 = 0, p1 = 0;
        if (valid) {
            p0 = j.ptr[k];
            p1 = j.ptr[k + 1];
        }
        bool ok = true;
        if (cnt) {
            ok = mbar_wait(&bar[s], (phase >> s) & 1u);
            phase ^= 1u << s;
        }
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicOr(j.err, DERR_TIMEOUT);
                unsigned ph = phase;
                for (int q = 0; q < 2; ++q)
                    if ((pending >> q) & 1u) {
                        // the stage that timed out already flipped its parity bit
                        unsigned want = (q == s) ? (((ph >> q) & 1u) ^ 1u) : ((ph >> q) & 1u);
                        mbar_wait(&bar[q], want);
                    }
            }
            __syncthreads();
            return;
        }
        if (threadIdx.x == 0 && cnt) pending &= ~(1u << s);
        T acc = T(0);
        if (cnt) {
            const int *sc = s_col[s];
            const T *sv = s_val[s];
#pragma unroll 4
            for (int p = p0 + g; p < p1; p += G) acc += sv[p - a0] * j.in[sc[p - a0]];
        } else {
            for (int p = p0 + g; p < p1; p += G) acc += __ldcs(j.val + p) * j.in[__ldcs(j.col + p)];
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o, G);
        if (valid && g == 0) {
            if (MODE == RESTRICT) {
                j.out[k] = acc + j.in[j.cpts[k]];
            } else {
                const int i = j.srow[k];
                if (!j.active || j.active[j.rowdir[i]]) {
                    const T v = j.in[i] + j.dinv[i] * (j.b[i] - acc);
                    if (MODE == C_SWEEP_FINAL) {
                        j.x64[i] += (double)v;
                    } else {
                        j.out[i] = v;
                        if (MODE == F_SWEEP && j.x64) j.x64[i] += (double)v;
                    }
                }
            }
        }
        __syncthreads();   // stage s is free again
        if (threadIdx.x == 0) issue(t + 2 * gridDim.x, s);
    }
}

}  // namespace tile
}  // namespace pr
