// AIR V-cycle on the GPU (Sec. 1.2; relaxation Sec. 2 and Sec. 4: pointwise
// Jacobi).  Correction form with zero initial guess on every level:
//   level 0: r = b - A x (FP64, cast to the cycle precision T), per-matrix ||r||
//   down:    b_{l+1} = R_l b_l, R row = [Z_i, 1] (restriction of the residual)
//   coarsest: coarse_sweeps Jacobi sweeps from 0 (one CTA per matrix segment)
//   up:      y_l = P x_{l+1} (one-point: y_i = x_{l+1}[pmap(i)])
//            F rows: xn = y + D^{-1}(b - A y);  C rows: xn = y
//            C rows: x = xn + D^{-1}(b - A xn); F rows: x = xn   (level 0: x_FP64 += x)
// Level 0 of the structured hex operator is stored in block form (identity
// diagonal implicit, three 8 x 4 face blocks per element, 16-byte row loads);
// coarse levels are CSR with a group of G lanes per row.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include "common.cuh"

namespace pr {

namespace {

constexpr int BS = 256;

// Timing event: a plain record, or an event-record node while the stream is
// being captured into a graph (so each replay records it).
void rec_event(cudaEvent_t e, cudaStream_t s) {
    cudaStreamCaptureStatus cs;
    PR_CUDA(cudaStreamIsCapturing(s, &cs));
    if (cs == cudaStreamCaptureStatusActive) PR_CUDA(cudaEventRecordWithFlags(e, s, cudaEventRecordExternal));
    else PR_CUDA(cudaEventRecord(e, s));
}

__device__ __forceinline__ int face_node(int d, int o, int t) {
    return d == 0 ? (o | (t << 1)) : d == 1 ? ((t & 1) | (o << 1) | ((t >> 1) << 2)) : (t | (o << 2));
}

template <class T>
struct V4 {
    T x, y, z, w;
};

// block values are read once per sweep: streaming loads (evict-first), so the
// vectors gathered by the face terms stay in L2
__device__ __forceinline__ V4<float> load4(const float *p) {
    float4 v = __ldcs(reinterpret_cast<const float4 *>(p));
    return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ V4<double> load4(const double *p) {
    double2 a = __ldcs(reinterpret_cast<const double2 *>(p));
    double2 b = __ldcs(reinterpret_cast<const double2 *>(p) + 1);
    return {a.x, a.y, b.x, b.y};
}

// Off-diagonal part of row (m, e, a) of the hex block operator applied to v
// (v points at direction m's vector).  Returns sum_faces sum_t A v.
// Level-0 block kernels run on a 3-D grid: x = tiles of 32 elements along a
// mesh row (8 rows each, 256 threads), y = iy + n iz, z = direction, so the
// element coordinates come from block indices.
struct HexRow {
    int m, e, a, idx[3];
    bool valid;
};

__device__ __forceinline__ HexRow hex_row(int n) {
    HexRow r;
    r.m = blockIdx.z;
    int ix = blockIdx.x * 32 + (threadIdx.x >> 3);
    r.a = threadIdx.x & 7;
    r.idx[0] = ix;
    r.idx[1] = blockIdx.y % n;
    r.idx[2] = blockIdx.y / n;
    r.valid = ix < n;
    r.e = ix + n * (int)blockIdx.y;
    return r;
}

template <class T, class TV>
__device__ __forceinline__ T bsr_offdiag(int n, long long E, int m, int e, int a, const int *idx, const int8_t *dsign,
                                         const T *vals, const TV *v) {
    const int stride[3] = {1, n, n * n};
    T acc = T(0);
    const T *base = vals + (((long long)m * E + e) * 3) * 32 + a * 4;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        int sg = dsign[3 * m + d];
        if (sg == 0) continue;
        bool has = sg > 0 ? idx[d] > 0 : idx[d] < n - 1;
        if (!has) continue;
        int ep = sg > 0 ? e - stride[d] : e + stride[d];
        int o = sg > 0 ? 1 : 0;
        V4<T> w = load4(base + d * 32);
        const TV *xb = v + 8LL * ep;
        acc += w.x * (T)xb[face_node(d, o, 0)];
        acc += w.y * (T)xb[face_node(d, o, 1)];
        acc += w.z * (T)xb[face_node(d, o, 2)];
        acc += w.w * (T)xb[face_node(d, o, 3)];
    }
    return acc;
}

// Block sum of per-thread FP32 squares: FP32 inside each warp, one conversion
// per warp, FP64 across warps (fixed order).
__device__ __forceinline__ double block_sum_f(float v) {
    __shared__ double shf[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) shf[w] = (double)v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        int nw = (blockDim.x + 31) >> 5;
        for (int k = 0; k < nw; ++k) s += shf[k];
    }
    __syncthreads();
    return s;
}

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sh[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        int nw = (blockDim.x + 31) >> 5;
        for (int k = 0; k < nw; ++k) s += sh[k];
    }
    __syncthreads();
    return s;
}

// ---- level-0 FP64 residual --------------------------------------------------
template <class T>
__global__ void __launch_bounds__(BS) k_res0_bsr(int n, int N, const int8_t *dsign, const double *bsr64,
                                                 const double *b, const double *x, T *r, float *r2,
                                                 double *partials, int maxblk, const int *active, int zero_x) {
    pdl_begin();
    HexRow q = hex_row(n);
    if (active && !active[q.m]) return;
    constexpr bool F32 = std::is_same<T, float>::value;
    double s2 = 0.0;
    float s2f = 0.0f;
    long long E = (long long)N / 8;
    if (q.valid) {
        long long gi = (long long)q.m * N + 8LL * q.e + q.a;
        // x = 0 (a solve's first residual): r = b, no operator read
        double acc = b[gi];
        if (!zero_x) {
            acc -= x[gi];
            acc -= bsr_offdiag<double, double>(n, E, q.m, q.e, q.a, q.idx, dsign, bsr64, x + (long long)q.m * N);
        }
        T rt = (T)acc;
        r[gi] = rt;
        if (r2) r2[gi] = (float)rt;   // the inner iteration's fixed right-hand side
        // the stopping test needs ||r|| to a few digits: with an FP32 cycle the
        // square of the cast value is summed in FP32 inside each warp
        if (F32) s2f = (float)rt * (float)rt;
        else s2 = acc * acc;
    }
    double tot = F32 ? block_sum_f(s2f) : block_sum(s2);
    if (threadIdx.x == 0) partials[(long long)q.m * maxblk + blockIdx.y * gridDim.x + blockIdx.x] = tot;
}

// ---- double-float arithmetic (error-free transformations) -----------------------
// A value is the unevaluated sum hi + lo of two floats.  two_sum (Knuth) returns
// s = fl(a + b) and the exact error; fast_two_sum (Dekker) assumes |a| >= |b|; the
// exact error of a product comes from one fma.  Products of pairs drop lo*lo
// (below 2^-48 relative).  With these, r = b - x - A x keeps about 44 bits, far
// below the 1e-8 relative residuals the refinement resolves, on the FP32 pipe.
__device__ __forceinline__ float2 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return make_float2(s, e);
}
__device__ __forceinline__ float2 fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}
// acc += a * x, all pairs
__device__ __forceinline__ void dd_fma_acc(float2 &acc, float2 a, float2 x) {
    const float p = __fmul_rn(a.x, x.x);
    const float pe = __fmaf_rn(a.x, x.x, -p);
    const float t = __fmaf_rn(a.x, x.y, __fmaf_rn(a.y, x.x, pe));
    const float2 s2 = two_sum(acc.x, p);
    acc.x = s2.x;
    acc.y = __fadd_rn(acc.y, __fadd_rn(s2.y, t));
}
__device__ __forceinline__ float2 dd_split(double d) {
    const float hi = __double2float_rn(d);
    return make_float2(hi, __double2float_rn(d - (double)hi));
}

__device__ __forceinline__ void load_dd4(const float2 *p, float2 *w) {
    const float4 a = __ldcs(reinterpret_cast<const float4 *>(p));
    const float4 b = __ldcs(reinterpret_cast<const float4 *>(p) + 1);
    w[0] = make_float2(a.x, a.y);
    w[1] = make_float2(a.z, a.w);
    w[2] = make_float2(b.x, b.y);
    w[3] = make_float2(b.z, b.w);
}

// Level-0 residual of the block form in double-float: r = b - x - sum_faces A x_nbr,
// cast to FP32 for the cycle, FP32 squares for the norm (as in k_res0_bsr<float>)
__global__ void __launch_bounds__(BS) k_res0_bsr_dd(int n, int N, const int8_t *dsign, const float2 *vals,
                                                    const float2 *b, const float2 *x, float *r, float *r2,
                                                    double *partials, int maxblk, const int *active) {
    pdl_begin();
    HexRow q = hex_row(n);
    if (active && !active[q.m]) return;
    float s2f = 0.0f;
    if (q.valid) {
        const long long E = (long long)N / 8;
        const long long gi = (long long)q.m * N + 8LL * q.e + q.a;
        const float2 bi = b[gi], xi = x[gi];
        const float2 *xm = x + (long long)q.m * N;
        const int stride[3] = {1, n, n * n};
        const float2 *base = vals + (((long long)q.m * E + q.e) * 3) * 32 + q.a * 4;
        float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int sg = dsign[3 * q.m + d];
            if (sg == 0) continue;
            const bool has = sg > 0 ? q.idx[d] > 0 : q.idx[d] < n - 1;
            if (!has) continue;
            const int ep = sg > 0 ? q.e - stride[d] : q.e + stride[d];
            const int o = sg > 0 ? 1 : 0;
            float2 w[4];
            load_dd4(base + d * 32, w);
            const float2 *xb = xm + 8LL * ep;
#pragma unroll
            for (int t = 0; t < 4; ++t) dd_fma_acc(acc, w[t], xb[face_node(d, o, t)]);
        }
        acc = fast_two_sum(acc.x, acc.y);
        // (b - x) - acc in pairs
        float2 d0 = two_sum(bi.x, -xi.x);
        d0.y = __fadd_rn(d0.y, __fsub_rn(bi.y, xi.y));
        const float2 d1 = two_sum(d0.x, -acc.x);
        const float lo = __fadd_rn(__fsub_rn(d0.y, acc.y), d1.y);
        const float rt = __fadd_rn(d1.x, lo);
        r[gi] = rt;
        if (r2) r2[gi] = rt;
        s2f = rt * rt;
    }
    const double tot = block_sum_f(s2f);
    if (threadIdx.x == 0) partials[(long long)q.m * maxblk + blockIdx.y * gridDim.x + blockIdx.x] = tot;
}

__global__ void k_dd_split(long long n, const double *a, float2 *out) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = dd_split(a[i]);
}

__global__ void k_dd_join(long long n, const float2 *a, double *out) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (double)a[i].x + (double)a[i].y;
}

template <class T>
__global__ void __launch_bounds__(BS) k_res0_csr(const int *row0, const int *nrow, const int *rowptr, const int *col,
                                                 const double *val, const double *b, const double *x, T *r,
                                                 float *r2, double *partials, int maxblk, const int *active,
                                                 int zero_x) {
    pdl_begin();
    int m = blockIdx.y;
    if (active && !active[m]) return;
    int li = blockIdx.x * blockDim.x + threadIdx.x;
    double s2 = 0.0;
    if (li < nrow[m]) {
        int i = row0[m] + li;
        double acc = 0.0;
        if (!zero_x)   // x = 0 (a solve's first residual): r = b, no operator read
            for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) acc += val[p] * x[col[p]];
        acc = b[i] - acc;
        r[i] = (T)acc;
        if (r2) r2[i] = (float)acc;
        s2 = acc * acc;
    }
    double tot = block_sum(s2);
    if (threadIdx.x == 0) partials[(long long)m * maxblk + blockIdx.x] = tot;
}

// ---- inner correction (FP32) ---------------------------------------------------
// A refinement step solves A d = r (r = the outer residual, cast to FP32 in r32)
// by FP32 V-cycles; between cycles the FP32 residual r32 - A d32 is the next
// cycle's right-hand side.  Block form: identity diagonal, element-ordered FP32
// face blocks (bsr32), the same grid and norm partials as the outer residual.
__global__ void __launch_bounds__(BS) k_res32_bsr(int n, int N, const int8_t *dsign, const float *bsr32,
                                                  const float *r0, const float *d, float *r, double *partials,
                                                  int maxblk, const int *active) {
    pdl_begin();
    HexRow q = hex_row(n);
    if (active && !active[q.m]) return;
    float s2f = 0.0f;
    if (q.valid) {
        const long long E = (long long)N / 8;
        const long long gi = (long long)q.m * N + 8LL * q.e + q.a;
        const float r0i = r0[gi], di = d[gi];
        const float acc = bsr_offdiag<float, float>(n, E, q.m, q.e, q.a, q.idx, dsign, bsr32, d + (long long)q.m * N);
        const float rt = r0i - (di + acc);
        r[gi] = rt;
        s2f = rt * rt;
    }
    const double tot = block_sum_f(s2f);
    if (threadIdx.x == 0) partials[(long long)q.m * maxblk + blockIdx.y * gridDim.x + blockIdx.x] = tot;
}

// CSR level 0 (diagonal stored): r = r0 - A d with FP32 values
__global__ void __launch_bounds__(BS) k_res32_csr(const int *row0, const int *nrow, const int *rowptr, const int *col,
                                                  const float *val, const float *r0, const float *d, float *r,
                                                  double *partials, int maxblk, const int *active) {
    pdl_begin();
    const int m = blockIdx.y;
    if (active && !active[m]) return;
    const int li = blockIdx.x * blockDim.x + threadIdx.x;
    float s2f = 0.0f;
    if (li < nrow[m]) {
        const int i = row0[m] + li;
        float acc = 0.0f;
        for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) acc += val[p] * d[col[p]];
        const float rt = r0[i] - acc;
        r[i] = rt;
        s2f = rt * rt;
    }
    const double tot = block_sum_f(s2f);
    if (threadIdx.x == 0) partials[(long long)m * maxblk + blockIdx.x] = tot;
}


// Step norms: one CTA per matrix.  Thread t sums the matrix's partials t, t +
// NORM_BS, ... in order, then a fixed tree (deterministic); every CTA then takes a
// ticket, and the last one sets *any from the flags of all matrices.
constexpr int NORM_BS = 256;

__device__ __forceinline__ double cta_sum_partials(const double *p, int cnt) {
    __shared__ double sh[NORM_BS];
    double s = 0.0;
    for (int k = threadIdx.x; k < cnt; k += NORM_BS) s += p[k];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int h = NORM_BS / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

__device__ __forceinline__ void any_from_last_cta(int ndir, const int *flags, int *any, unsigned *ticket) {
    __shared__ bool last;
    __threadfence();   // this CTA's flag before its ticket
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == (unsigned)ndir - 1u;
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        int a = 0;
        for (int d = 0; d < ndir; ++d) a |= ((volatile const int *)flags)[d];
        *any = a;
        *ticket = 0u;
    }
}

// outer norm of a step: ||r||, active (||r|| > tol ||b||), and the step's inner flag
// and threshold; *any = 1 if a matrix takes part in the step
__global__ void __launch_bounds__(NORM_BS) k_norm_outer(int ndir, const double *partials, int maxblk, double *out,
                                                        const double *bnorm, double tol, int *active, int *iactive,
                                                        double *ithr, int *any, unsigned *ticket) {
    pdl_begin();
    const int m = blockIdx.x;
    const int was = active[m];   // converged earlier: its partials were not written
    if (was) {
        const double nr = sqrt(cta_sum_partials(partials + (long long)m * maxblk, maxblk));
        if (threadIdx.x == 0) {
            out[m] = nr;
            const int a = nr > tol * bnorm[m] ? 1 : 0;
            active[m] = a;
            iactive[m] = a;
            ithr[m] = fmax(INNER_TOL_FRAC * tol * bnorm[m], INNER_ETA * nr);
        }
    } else if (threadIdx.x == 0) {
        iactive[m] = 0;
    }
    any_from_last_cta(ndir, iactive, any, ticket);
}

// inner norm after a cycle: counts the cycle (icount accumulates over a solve) and
// clears the inner flag once the FP32 residual reaches the step's threshold; *any =
// 1 while a matrix still cycles
__global__ void __launch_bounds__(NORM_BS) k_norm_inner(int ndir, const double *partials, int maxblk, double *out,
                                                        const double *ithr, int *iactive, int *icount, int *any,
                                                        unsigned *ticket) {
    pdl_begin();
    const int m = blockIdx.x;
    if (iactive[m]) {
        const double nr = sqrt(cta_sum_partials(partials + (long long)m * maxblk, maxblk));
        if (threadIdx.x == 0) {
            out[m] = nr;
            icount[m] += 1;
            iactive[m] = nr > ithr[m] ? 1 : 0;
        }
    }
    any_from_last_cta(ndir, iactive, any, ticket);
}

// end of a step: x += d on the rows of the matrices that took part (d cleared);
// the iterate is FP64 or, in double-float mode, a float pair
// (every load is issued before the stores: a load behind a store to a pointer that
// may alias it waits for that store to complete)
__global__ void k_fold_delta(const int *row0, const int *nrow, float *__restrict__ d, double *__restrict__ x64,
                             float2 *__restrict__ xdd, const int *active) {
    pdl_begin();
    const int m = blockIdx.y;
    if (!active[m]) return;
    const int li = blockIdx.x * blockDim.x + threadIdx.x;
    if (li >= nrow[m]) return;
    const long long i = (long long)row0[m] + li;
    const float v = d[i];
    if (xdd) {
        const float2 xo = xdd[i];
        const float2 s2 = two_sum(xo.x, v);
        d[i] = 0.0f;
        xdd[i] = fast_two_sum(s2.x, __fadd_rn(xo.y, s2.y));
    } else {
        const double xo = x64[i];
        d[i] = 0.0f;
        x64[i] = xo + (double)v;
    }
}

__global__ void k_to_f32(long long n, const double *a, float *out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)a[i];
}

// per-matrix norm from the partials: a warp per matrix, lane k sums partials
// k, k+32, ... in order, then a fixed shuffle tree (deterministic)
__global__ void k_norm_final(int ndir, const double *partials, int maxblk, double *out, const double *bnorm,
                             double tol, int *active) {
    pdl_begin();
    int m = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    int lane = threadIdx.x & 31;
    if (m >= ndir) return;
    if (active && !active[m]) return;
    double s = 0.0;
    for (int k = lane; k < maxblk; k += 32) s += partials[(long long)m * maxblk + k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        double nr = sqrt(s);
        out[m] = nr;
        if (active && bnorm) active[m] = nr > tol * bnorm[m] ? 1 : 0;
    }
}

// F32: squares of the values cast to FP32, summed in FP32 inside each warp (a norm
// for a stopping test, without the narrow FP64 pipe); else FP64 throughout
template <bool F32>
__global__ void k_sumsq_rows(const int *row0, const int *nrow, const double *v, double *partials, int maxblk) {
    int m = blockIdx.y;
    int li = blockIdx.x * blockDim.x + threadIdx.x;
    double s2 = 0.0;
    float s2f = 0.0f;
    if (li < nrow[m]) {
        double a = v[row0[m] + li];
        if (F32) s2f = (float)a * (float)a;
        else s2 = a * a;
    }
    double tot = F32 ? block_sum_f(s2f) : block_sum(s2);
    if (threadIdx.x == 0) partials[(long long)m * maxblk + blockIdx.x] = tot;
}

// ---- sparse row dot products on SELL copies --------------------------------------
// One thread per row.  The coarse sweeps are latency-bound (dependent loads per
// thread), so a thread issues the loads of SELL_U entries together, then their
// SELL_U gathers, and only then adds; entry addresses need nothing but the slice
// offset, and a warp's loads of one entry index are one contiguous 128-byte line.
// Entries are streamed (evict-first) so the gathered vector stays in L2.  Terms are
// added in ascending entry order.
constexpr int SELL_U = 8;

template <class T, int G, int U>
__device__ __forceinline__ T sell_dot(int base, int len, int g, const int *col, const T *val, const T *in) {
    T acc = T(0);
    for (int j0 = g; j0 < len; j0 += U * G) {
        int c[U];
        T v[U], x[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const bool ok = j0 + u * G < len;
            c[u] = ok ? __ldcs(col + base + 32 * (j0 + u * G)) : 0;
            v[u] = ok ? __ldcs(val + base + 32 * (j0 + u * G)) : T(0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) x[u] = j0 + u * G < len ? in[c[u]] : T(0);
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (j0 + u * G < len) acc += v[u] * x[u];
    }
    return acc;
}

// the same with 16-bit column offsets from the row r (col = r + offset)
template <class T, int G, int U>
__device__ __forceinline__ T sell_dot16(int base, int len, int g, int r, const short *col16, const T *val,
                                        const T *in) {
    T acc = T(0);
    for (int j0 = g; j0 < len; j0 += U * G) {
        int c[U];
        T v[U], x[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const bool ok = j0 + u * G < len;
            c[u] = ok ? r + (int)__ldcs(col16 + base + 32 * (j0 + u * G)) : 0;
            v[u] = ok ? __ldcs(val + base + 32 * (j0 + u * G)) : T(0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) x[u] = j0 + u * G < len ? in[c[u]] : T(0);
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (j0 + u * G < len) acc += v[u] * x[u];
    }
    return acc;
}


enum SellMode : int { SM_F = 0, SM_C = 1, SM_C_FINAL = 2, SM_RESTRICT = 3 };

// entries per lane issued together: SELL_U for the sweeps; the restriction's short
// rows (6-9 entries) take SELL_U / G, so a row's G lanes together still cover SELL_U
// entries per pass without predicated-off slots (the same for the sweeps measured no
// faster)
template <int MODE, int G>
constexpr int sell_unroll() {
    return MODE == SM_RESTRICT ? (SELL_U / G > 1 ? SELL_U / G : 1) : SELL_U;
}

template <class T>
struct SellJob {
    int npos;
    const int *ptr, *row, *len, *col;
    const short *col16;   // 16-bit column offsets from the row (restriction: from its coarse
                          // point's fine row); col is then null
    const T *val;
    const T *in;          // vector the rows multiply
    const T *dinv, *b;    // sweeps
    T *out;
    double *x64;          // F sweep: optional fold; final C sweep: target
    float *d32;           // inner correction: fold / final target instead of x64
    const int *cpts;      // restriction: fine row of each coarse point
    const int *active, *rowdir;
    const int *any;       // inner correction: the launch does nothing once *any == 0
};

// F sweep:   out[i] = in[i] + dinv[i] (b[i] - A_i in)        (x64[i] += it, if given)
// C sweep:   same into out, or (final) x64[i] += it
// restrict:  out[ic] = Z_ic in + in[cpts[ic]]
// G lanes per row (G > 1 on small levels, where rows are too few to fill the GPU):
// lane g takes entries g, g+G, ..., then a fixed shuffle tree; the launch covers
// exactly npos * G threads (npos is a multiple of 256), so every lane reaches the
// shuffles.
template <class T, int MODE, int G>
__global__ void __launch_bounds__(BS) k_sell(SellJob<T> j) {
    pdl_begin();
    if (j.any && !*j.any) return;
    const long long t = (long long)blockIdx.x * BS + threadIdx.x;
    const int q = (int)(t / G), g = (int)(t % G);
    const int r = j.row[q];
    bool ok = r >= 0;
    if (MODE != SM_RESTRICT && ok && j.active && !j.active[j.rowdir[r]]) ok = false;
    const int len = ok ? j.len[q] : 0;
    const int base = j.ptr[q >> 5] + (q & 31);
    // the row's own operands are loaded before the dot product (shorter chain); a
    // restriction row's 16-bit columns are offsets from its coarse point's fine row
    T own = T(0), di = T(0), bi = T(0);
    const int rb = (MODE == SM_RESTRICT && ok && j.col16) ? j.cpts[r] : r;
    if (ok && g == 0) {
        if (MODE == SM_RESTRICT) {
            own = j.in[j.col16 ? rb : j.cpts[r]];
        } else {
            own = j.in[r];
            di = j.dinv[r];
            bi = j.b[r];
        }
    }
    constexpr int U = sell_unroll<MODE, G>();
    T acc = j.col16 ? sell_dot16<T, G, U>(base, len, g, rb, j.col16, j.val, j.in)
                    : sell_dot<T, G, U>(base, len, g, j.col, j.val, j.in);
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o, G);
    if (!ok || g != 0) return;
    if (MODE == SM_RESTRICT) {
        j.out[r] = acc + own;
        return;
    }
    const T v = own + di * (bi - acc);
    if (MODE == SM_C_FINAL) {
        if (j.d32) j.d32[r] += (float)v;
        else j.x64[r] += (double)v;
    } else {
        // the fold's load before the store to out
        if (MODE == SM_F && j.d32) j.d32[r] += (float)v;
        else if (MODE == SM_F && j.x64) j.x64[r] += (double)v;
        j.out[r] = v;
    }
}

// ---- prolongation y = P x_c --------------------------------------------------
// The coarse vector of level l+1 lives in two buffers after its relaxation: F rows
// in xcF, C and coarsest rows in xc.  C rows of y are also written to y2 (the other
// ping-pong buffer of the F sweeps), so the F sweeps never copy C rows.
template <class T>
__device__ __forceinline__ void prolong_row(long long i, int8_t c, int p, const int8_t *cfc, const T *xcF,
                                            const T *xc, T *y, T *y2) {
    if (c == CF_COARSEST) return;
    T v = T(0);
    if (p >= 0) {
        // both candidates are loaded with the flag (one dependent step, not two)
        const int8_t cc = cfc[p];
        const T vf = xcF[p], vc = xc[p];
        v = cc == CF_F ? vf : vc;
    }
    y[i] = v;
    if (y2 && c == CF_C) y2[i] = v;
}

// four consecutive rows per thread (vector loads of cf and pmap, twelve gathers in
// flight): with one row per thread the kernel is latency-bound
template <class T>
__global__ void k_prolong(int n, const int8_t *cf, const int *pmap, const int8_t *cfc, const T *xcF, const T *xc,
                          T *y, T *y2, const int *any) {
    pdl_begin();
    if (any && !*any) return;
    const long long i0 = 4LL * ((long long)blockIdx.x * blockDim.x + threadIdx.x);
    if (i0 >= n) return;
    if (i0 + 4 <= n) {
        const char4 c4 = *reinterpret_cast<const char4 *>(cf + i0);
        const int4 p4 = *reinterpret_cast<const int4 *>(pmap + i0);
        const int8_t c[4] = {(int8_t)c4.x, (int8_t)c4.y, (int8_t)c4.z, (int8_t)c4.w};
        const int p[4] = {p4.x, p4.y, p4.z, p4.w};
        int8_t cc[4];
        T vf[4], vc[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const bool gth = c[u] != CF_COARSEST && p[u] >= 0;
            cc[u] = gth ? cfc[p[u]] : (int8_t)CF_C;
            vf[u] = gth ? xcF[p[u]] : T(0);
            vc[u] = gth ? xc[p[u]] : T(0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (c[u] == CF_COARSEST) continue;
            const T v = cc[u] == CF_F ? vf[u] : vc[u];
            y[i0 + u] = v;
            if (y2 && c[u] == CF_C) y2[i0 + u] = v;
        }
    } else {
        for (long long i = i0; i < n; ++i) prolong_row<T>(i, cf[i], pmap[i], cfc, xcF, xc, y, y2);
    }
}

// single-level hierarchies: x64 += the coarsest solution on active rows
template <class T>
__global__ void k_fold_coarsest(int n, const T *xco, double *x64, float *d32, float2 *xdd, const int *active,
                                const int *rowdir) {
    pdl_begin();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || (active && !active[rowdir[i]])) return;
    if (d32) {
        d32[i] += (float)xco[i];
    } else if (xdd) {
        const float2 xo = xdd[i];
        const float2 s2 = two_sum(xo.x, (float)xco[i]);
        xdd[i] = fast_two_sum(s2.x, __fadd_rn(xo.y, s2.y));
    } else {
        x64[i] += (double)xco[i];
    }
}

// first coarsest Jacobi sweep from x = 0 on the coarsest rows of the split (positions
// [kX, n)): x = D^{-1} b, the value x + D^{-1}(b - A x) takes at x = 0 (zero: no
// sweep, x = 0)
template <class T>
__global__ void k_jacobi0(int kX, int n, const int *srow, const T *dinv, const T *b, T *x, int zero,
                          const int *any) {
    pdl_begin();
    if (any && !*any) return;
    const long long p = kX + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int i = srow[p];
    x[i] = zero ? T(0) : dinv[i] * b[i];
}

// final correction at a CSR level 0: x64 += the coarsest solution on the rows of
// matrices that end there (split positions [kX, n))
template <class T>
__global__ void k_fold_split(int kX, int n, const int *srow, const T *xco, double *x64, float *d32,
                             const int *active, const int *rowdir, float2 *xdd, const int *any) {
    pdl_begin();
    if (any && !*any) return;
    int k = kX + blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int i = srow[k];
    if (active && !active[rowdir[i]]) return;
    if (d32) {
        d32[i] += (float)xco[i];
    } else if (xdd) {
        const float2 xo = xdd[i];
        const float2 s2 = two_sum(xo.x, (float)xco[i]);
        xdd[i] = fast_two_sum(s2.x, __fadd_rn(xo.y, s2.y));
    } else {
        x64[i] += (double)xco[i];
    }
}

// ---- BSR (hex level 0) relaxation, unit diagonal ------------------------------
template <class T, bool FINAL>
__global__ void __launch_bounds__(BS) k_relax_bsr(int n, int N, const int8_t *dsign, const T *vals, const int8_t *cf,
                                                  const T *b, const T *in, T *out, int phase, double *x64,
                                                  const T *xco, const int *active, float2 *xdd) {
    pdl_begin();
    HexRow q = hex_row(n);
    if (!q.valid) return;
    const long long gi = (long long)q.m * N + 8LL * q.e + q.a;
    // Loads that decide nothing are issued before any branch: the sweep is latency-
    // bound, and a load behind a branch on another load costs one more round trip.
    // The F sweeps (not final) also compute every row's face terms before knowing
    // whether the row is an F row (a C row's block values are then read for
    // nothing: a quarter of the rows, against one round trip saved for all).
    const int act = active ? active[q.m] : 1;
    const int8_t c = cf[gi];
    const T xin = in[gi], bi = b[gi];
    T acc = T(0);
    if (!FINAL)
        acc = bsr_offdiag<T, T>(n, (long long)N / 8, q.m, q.e, q.a, q.idx, dsign, vals, in + (long long)q.m * N);
    if (!act) return;
    T v = xin;
    if (c == CF_COARSEST) {   // a matrix whose hierarchy ends at level 0
        if (!FINAL) return;
        v = xco[gi];
    } else if (c == (phase == 0 ? CF_F : CF_C)) {
        if (FINAL)
            acc = bsr_offdiag<T, T>(n, (long long)N / 8, q.m, q.e, q.a, q.idx, dsign, vals,
                                    in + (long long)q.m * N);
        v = v + (bi - (acc + v));
    }
    if (!FINAL) {
        out[gi] = v;
    } else if (xdd) {   // iterate held as a float pair: x += v without the FP64 pipe
        const float2 xo = xdd[gi];
        const float2 s2 = two_sum(xo.x, (float)v);
        xdd[gi] = fast_two_sum(s2.x, __fadd_rn(xo.y, s2.y));
    } else {
        x64[gi] += (double)v;
    }
}

// ---- level-0 relaxation on the CF-split block copy (FP32) -------------------------
// One thread per row of the F (or C) group: the row's three face rows are read from
// v0 at its split position (contiguous across the group, so a sweep reads only its
// own rows' blocks), the row's element and node follow from its index.  x += v:
// a float pair (x_dd) or FP64.
__device__ __forceinline__ void x_add(long long gi, float v, float *d32, float2 *xdd, double *x64) {
    if (d32) {   // inner correction: the FP32 correction of the refinement step
        d32[gi] += v;
    } else if (xdd) {
        const float2 xo = xdd[gi];
        const float2 s2 = two_sum(xo.x, v);
        xdd[gi] = fast_two_sum(s2.x, __fadd_rn(xo.y, s2.y));
    } else {
        x64[gi] += (double)v;
    }
}

// rows at split positions [k0, k0 + cnt): F sweep (out, optional fold into x) or the
// final C sweep (into x)
template <bool FINAL>
__global__ void __launch_bounds__(BS) k_relax0_split(int n, int N, const int8_t *dsign, const int *srow, int k0,
                                                     int cnt, const float4 *v0, const float *b, const float *in,
                                                     float *out, bool fold, float *d32, float2 *xdd, double *x64,
                                                     const int *active, const int *any) {
    pdl_begin();
    if (any && !*any) return;
    const int k = blockIdx.x * BS + threadIdx.x;
    if (k >= cnt) return;
    const int gi = srow[k0 + k];
    const int m = gi / N;
    const int r = gi - m * N;
    const int e = r >> 3;   // the row's node is implicit in its face rows of v0
    const int ix = e % n, t = e / n, iy = t % n, iz = t / n;
    const int idx[3] = {ix, iy, iz};
    const int stride[3] = {1, n, n * n};
    const int act = active ? active[m] : 1;
    const float xin = in[gi], bi = b[gi];
    const float *xm = in + (long long)m * N;
    float acc = 0.0f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int sg = dsign[3 * m + d];
        if (sg == 0) continue;
        const bool has = sg > 0 ? idx[d] > 0 : idx[d] < n - 1;
        if (!has) continue;
        const int ep = sg > 0 ? e - stride[d] : e + stride[d];
        const int o = sg > 0 ? 1 : 0;
        const float4 w = __ldcs(v0 + 3LL * (k0 + k) + d);
        const float *xb = xm + 8LL * ep;
        acc += w.x * xb[face_node(d, o, 0)];
        acc += w.y * xb[face_node(d, o, 1)];
        acc += w.z * xb[face_node(d, o, 2)];
        acc += w.w * xb[face_node(d, o, 3)];
    }
    if (!act) return;
    const float v = xin + (bi - (acc + xin));
    if (!FINAL) {
        if (fold) x_add(gi, v, d32, xdd, x64);   // its load before the store to out
        out[gi] = v;
    } else {
        x_add(gi, v, d32, xdd, x64);
    }
}

// v0 from the element-ordered block form, by split position
__global__ void k_split0_copy(int nrows, int N, const int *srow, const float *bsr32, float4 *v0) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nrows) return;
    const int gi = srow[k];
    const long long m = gi / N;
    const int r = gi - (int)m * N;
    const int e = r >> 3, a = r & 7;
    const long long E = N / 8;
    const float *src = bsr32 + ((m * E + e) * 3) * 32 + a * 4;
#pragma unroll
    for (int d = 0; d < 3; ++d)
        v0[3LL * k + d] = make_float4(src[d * 32], src[d * 32 + 1], src[d * 32 + 2], src[d * 32 + 3]);
}

// ---- coarsest level: Jacobi sweeps, one CTA per matrix segment ---------------
// segment rows r0.. sit at split positions s0.. (the coarsest group of the split).
// A segment whose entries, vectors and row pointer fit CS_SMEM bytes is copied to
// shared memory once and swept there (each sweep of a global-memory segment is a
// chain of L2 round trips: 20 sweeps of a 31-row segment took ~15 us); columns are
// rebased to the segment, so the sums run in the same order and round alike.
// Levels with a larger segment sweep grid-wide on a SELL copy of their coarsest
// rows instead (coarsest_sell); the global-memory path below remains for segments
// whose columns leave the segment.

// The Jacobi sweeps of one segment by the whole CTA (sm: CS_SMEM bytes of shared
// memory, bad: one shared int)
template <class T>
__device__ void coarsest_seg(int r0, int nr, int s0, const int *sptr, const int *scol, const T *sval,
                             const T *dinv, const T *b, T *x, T *xt, int sweeps, unsigned char *sm, int *bad) {
    const int p0 = sptr[s0], nz = sptr[s0 + nr] - p0;
    const size_t need = (size_t)nz * (sizeof(T) + sizeof(int)) + 4 * (size_t)nr * sizeof(T) + (size_t)(nr + 1) * sizeof(int);
    if (need <= (size_t)CS_SMEM) {
        T *v = reinterpret_cast<T *>(sm);
        T *di = v + nz, *bb = di + nr, *c0 = bb + nr, *c1 = c0 + nr;
        int *ci = reinterpret_cast<int *>(c1 + nr), *rp = ci + nz;
        if (threadIdx.x == 0) *bad = 0;
        __syncthreads();
        for (int p = threadIdx.x; p < nz; p += blockDim.x) {
            const int c = scol[p0 + p] - r0;
            if (c < 0 || c >= nr) *bad = 1;   // not a whole-matrix segment: global path
            v[p] = sval[p0 + p];
            ci[p] = c;
        }
        for (int i = threadIdx.x; i <= nr; i += blockDim.x) rp[i] = sptr[s0 + i] - p0;
        for (int i = threadIdx.x; i < nr; i += blockDim.x) {
            di[i] = dinv[r0 + i];
            bb[i] = b[r0 + i];
            c0[i] = T(0);
        }
        __syncthreads();
        if (!*bad) {
            T *cur = c0, *nxt = c1;
            for (int sw = 0; sw < sweeps; ++sw) {
                for (int li = threadIdx.x; li < nr; li += blockDim.x) {
                    T acc = T(0);
                    for (int p = rp[li]; p < rp[li + 1]; ++p) acc += v[p] * cur[ci[p]];
                    nxt[li] = cur[li] + di[li] * (bb[li] - acc);
                }
                __syncthreads();
                T *t = cur; cur = nxt; nxt = t;
            }
            for (int li = threadIdx.x; li < nr; li += blockDim.x) x[r0 + li] = cur[li];
            return;
        }
    }
    for (int i = threadIdx.x; i < nr; i += blockDim.x) x[r0 + i] = T(0);
    __syncthreads();
    T *cur = x, *nxt = xt;
    for (int s = 0; s < sweeps; ++s) {
        for (int li = threadIdx.x; li < nr; li += blockDim.x) {
            int i = r0 + li, k = s0 + li;
            T acc = T(0);
            for (int p = sptr[k]; p < sptr[k + 1]; ++p) acc += sval[p] * cur[scol[p]];
            nxt[i] = cur[i] + dinv[i] * (b[i] - acc);
        }
        __syncthreads();
        T *t = cur; cur = nxt; nxt = t;
    }
    if (cur != x)
        for (int li = threadIdx.x; li < nr; li += blockDim.x) x[r0 + li] = cur[r0 + li];
}

template <class T>
__global__ void k_coarsest(const int *seg_row0, const int *seg_n, const int *seg_s0, const int *sptr,
                           const int *scol, const T *sval, const T *dinv, const T *b, T *x, T *xt, int sweeps,
                           const int *any) {
    pdl_begin();
    if (any && !*any) return;
    __shared__ __align__(16) unsigned char cs_sm[CS_SMEM];
    __shared__ int cs_bad;
    coarsest_seg<T>(seg_row0[blockIdx.x], seg_n[blockIdx.x], seg_s0[blockIdx.x], sptr, scol, sval, dinv, b, x, xt,
                    sweeps, cs_sm, &cs_bad);
}

template <class T>
const T *lv_dinv(const Level &L);
template <>
const float *lv_dinv<float>(const Level &L) { return L.dinv32; }
template <>
const double *lv_dinv<double>(const Level &L) { return L.dinv; }
template <class T, int MODE>
void launch_sell_g(const Sell &S, SellJob<T> j, int G, cudaStream_t s) {
    j.npos = S.npos;
    j.ptr = S.ptr;
    j.row = S.row;
    j.len = S.len;
    j.col = S.col;
    j.col16 = S.col16;
    j.val = (const T *)S.val;
    switch (G) {
        case 1: launch_pdl(k_sell<T, MODE, 1>, blocks_for(S.npos, BS), BS, s, j); break;
        case 2: launch_pdl(k_sell<T, MODE, 2>, blocks_for(2LL * S.npos, BS), BS, s, j); break;
        case 4: launch_pdl(k_sell<T, MODE, 4>, blocks_for(4LL * S.npos, BS), BS, s, j); break;
        default: launch_pdl(k_sell<T, MODE, 8>, blocks_for(8LL * S.npos, BS), BS, s, j); break;
    }
    PR_LAUNCH();
}

// lanes per row: the autotuner's choice, else enough threads to fill the GPU
// (about 2048 per SM) on small levels
int sell_lanes(const Sell &S, int sms) {
    if (S.G > 0) return S.G;
    const long long want = (long long)sms * 2048;
    int G = 1;
    while (G < 8 && (long long)S.npos * G * 2 <= want) G *= 2;
    return G;
}

template <class T, int MODE>
void launch_sell(const Sell &S, SellJob<T> j, int sms, cudaStream_t s) {
    if (S.nrows <= 0) return;
    launch_sell_g<T, MODE>(S, j, sell_lanes(S, sms), s);
}

// F sweep over the F rows (fold: x64 += the new values, the last level-0 sweep)
template <class T>
void relax_f(const Level &L, const T *b, const T *in, T *out, double *fold, float *fold32, const int *active,
             const int *any, int sms, cudaStream_t s) {
    SellJob<T> j{};
    j.any = any;
    j.in = in;
    j.dinv = lv_dinv<T>(L);
    j.b = b;
    j.out = out;
    j.x64 = fold;
    j.d32 = fold32;
    j.active = active;
    j.rowdir = L.rowdir;
    launch_sell<T, SM_F>(L.sF, j, sms, s);
}

// C sweep over the C rows into out, or (final) into x64 together with the coarsest
// rows of matrices that end on this level
template <class T>
void relax_c(const Level &L, const T *b, const T *in, T *out, double *x64, float *d32, const T *xco,
             const int *active, const int *any, int sms, cudaStream_t s) {
    SellJob<T> j{};
    j.any = any;
    j.in = in;
    j.dinv = lv_dinv<T>(L);
    j.b = b;
    j.out = out;
    j.x64 = x64;
    j.d32 = d32;
    j.active = active;
    j.rowdir = L.rowdir;
    if (x64 || d32) {
        launch_sell<T, SM_C_FINAL>(L.sC, j, sms, s);
        const int kX = L.nF + L.nC;
        if (L.n > kX) {
            launch_pdl(k_fold_split<T>, blocks_for(L.n - kX, BS), BS, s, kX, L.n, L.srow, xco, x64, d32, active,
                       L.rowdir, (float2 *)nullptr, any);
            PR_LAUNCH();
        }
    } else {
        launch_sell<T, SM_C>(L.sC, j, sms, s);
    }
}

// coarse_sweeps Jacobi sweeps from 0 over the coarsest rows of a level that has a
// SELL copy of them: the first is x = D^{-1} b, each further one a grid-wide SELL
// sweep; the buffers alternate so that the last sweep writes vx (which the
// prolongation and the level-0 fold read)
template <class T>
void coarsest_sell(const Level &L, int sweeps, const int *any, int sms, cudaStream_t s) {
    T *vx = (T *)L.vx, *vxn = (T *)L.vxn;
    const int kX = L.nF + L.nC;
    T *cur = (sweeps > 1 && (sweeps - 1) % 2 == 1) ? vxn : vx;
    launch_pdl(k_jacobi0<T>, blocks_for(L.n - kX, BS), BS, s, kX, L.n, L.srow, lv_dinv<T>(L), (const T *)L.vb, cur,
               sweeps == 0 ? 1 : 0, any);
    PR_LAUNCH();
    for (int k = 1; k < sweeps; ++k) {
        T *nxt = cur == vx ? vxn : vx;
        SellJob<T> j{};
        j.any = any;
        j.in = cur;
        j.dinv = lv_dinv<T>(L);
        j.b = (const T *)L.vb;
        j.out = nxt;
        j.rowdir = L.rowdir;
        launch_sell<T, SM_F>(L.sX, j, sms, s);
        cur = nxt;
    }
}

// b_c = Z b_F + b_C: one row of Z per coarse point
template <class T>
void restrict_(const Level &L, const T *bf, T *bc, const int *any, int sms, cudaStream_t s) {
    SellJob<T> j{};
    j.any = any;
    j.in = bf;
    j.out = bc;
    j.cpts = L.cpts;
    launch_sell<T, SM_RESTRICT>(L.sZ, j, sms, s);
}

// One V-cycle on lev[0].vb from a zero guess; its correction is added to x64 (the
// FP64 iterate, or the float-pair iterate in double-float mode) or, in the inner
// correction, to d32.  'active' gates the level-0 kernels per matrix; 'ps' (may be
// null) receives the level-0 and coarse-level relaxation events.
template <class T>
void vcycle_t(Hier &h, double *x64, float *d32, const int *active, ProfSlot *ps) {
    cudaStream_t s = h.stream;
    int NL = (int)h.lev.size();
    const bool prof = h.timed && ps;
    const int *any = d32 ? h.iany : nullptr;
    if (ps) ps->relax_timed = false;
    for (int l = 0; l < NL; ++l) {
        Level &L = h.lev[l];
        L.vF = L.vx;   // replaced by the F sweeps' buffer once the level relaxes
        if (l + 1 < NL) {
            const bool tr = prof && (int)ps->lvt.size() >= 4 * (l + 1);
            if (tr) rec_event(ps->lvt[4 * l], s);
            restrict_<T>(L, (const T *)L.vb, (T *)h.lev[l + 1].vb, any, h.sms, s);
            if (tr) rec_event(ps->lvt[4 * l + 1], s);
        }
        if (L.n_cseg && L.sX.nrows > 0) {
            const bool tx = prof && l >= 1 && (int)ps->lvx.size() >= 2 * (l + 1);
            if (tx) rec_event(ps->lvx[2 * l], s);
            coarsest_sell<T>(L, h.prm.coarse_sweeps, any, h.sms, s);
            if (tx) rec_event(ps->lvx[2 * l + 1], s);
        } else if (L.n_cseg) {
            launch_pdl(k_coarsest<T>, L.n_cseg, 256, s, L.d_cseg_row0, L.d_cseg_n, L.d_cseg_s0, L.sptr, L.scol,
                                                   (const T *)L.sval, lv_dinv<T>(L), (const T *)L.vb, (T *)L.vx,
                                                   (T *)L.vxn, h.prm.coarse_sweeps, any);
            PR_LAUNCH();
        }
    }
    const int fs = h.prm.f_sweeps;
    float2 *xdd = (h.dd && !d32) ? h.x_dd : nullptr;
    for (int l = NL - 2; l >= 0; --l) {
        Level &L = h.lev[l];
        const Level &C = h.lev[l + 1];
        const bool bsr = l == 0 && h.bsr0;
        // F sweeps ping-pong between vy and vxn; the C sweep reads the last one
        T *bufs[2] = {(T *)L.vy, (T *)L.vxn};
        const bool split0 = bsr && h.split0 && std::is_same<T, float>::value;
        const bool tp = prof && (int)ps->lvt.size() >= 4 * (l + 1);
        if (tp) rec_event(ps->lvt[4 * l + 2], s);
        launch_pdl(k_prolong<T>, blocks_for((L.n + 3) / 4, BS), BS, s, L.n, L.cf, L.pmap, C.cf, (const T *)C.vF,
                   (const T *)C.vx, bufs[0], (bsr && !split0) ? nullptr : bufs[1], any);
        PR_LAUNCH();
        if (tp) rec_event(ps->lvt[4 * l + 3], s);
        int cur = 0;
        if (split0) {
            // F sweeps over the F rows (the last one folds into x), C sweep over the C rows,
            // then the rows of matrices that end at level 0
            const int N = h.n0[0];
            const int kX = L.nF + L.nC;
            if (prof) { rec_event(ps->relax0[0], s); ps->relax_timed = true; }
            for (int f = 0; f < fs; ++f, cur ^= 1)
                if (L.nF > 0) {
                    launch_pdl(k_relax0_split<false>, blocks_for(L.nF, BS), BS, s, h.hex_n, N, h.dsign, L.srow, 0,
                               L.nF, h.v0, (const float *)L.vb, (const float *)bufs[cur], (float *)bufs[cur ^ 1],
                               f == fs - 1, d32, xdd, x64, active, any);
                    PR_LAUNCH();
                }
            if (L.nC > 0) {
                launch_pdl(k_relax0_split<true>, blocks_for(L.nC, BS), BS, s, h.hex_n, N, h.dsign, L.srow, L.nF,
                           L.nC, h.v0, (const float *)L.vb, (const float *)bufs[cur], (float *)nullptr, true, d32,
                           xdd, x64, active, any);
                PR_LAUNCH();
            }
            if (L.n > kX) {
                launch_pdl(k_fold_split<T>, blocks_for(L.n - kX, BS), BS, s, kX, L.n, L.srow, (const T *)L.vx, x64,
                           d32, active, L.rowdir, xdd, any);
                PR_LAUNCH();
            }
            if (prof) rec_event(ps->relax0[1], s);
        } else if (bsr) {
            int N = h.n0[0];
            dim3 grid(blocks_for(h.hex_n, 32), h.hex_n * h.hex_n, h.ndir);
            const T *vals = std::is_same<T, float>::value ? (const T *)h.bsr32 : (const T *)h.bsr64;
            if (prof) { rec_event(ps->relax0[0], s); ps->relax_timed = true; }
            for (int f = 0; f < fs; ++f, cur ^= 1) {
                launch_pdl(k_relax_bsr<T, false>, grid, BS, s, h.hex_n, N, h.dsign, vals, L.cf, (const T *)L.vb, bufs[cur],
                                                          bufs[cur ^ 1], 0, nullptr, nullptr, active, nullptr);
                PR_LAUNCH();
            }
            launch_pdl(k_relax_bsr<T, true>, grid, BS, s, h.hex_n, N, h.dsign, vals, L.cf, (const T *)L.vb, bufs[cur],
                                                     nullptr, 1, x64, (const T *)L.vx, active, xdd);
            PR_LAUNCH();
            if (prof) rec_event(ps->relax0[1], s);
        } else {
            // C rows stay where the prolongation put them (both buffers); F rows end in
            // bufs[cur], C rows in vx (level 0: both folded into the iterate instead)
            const int *act = l == 0 ? active : nullptr;
            bool tl = prof && l >= 1 && (int)ps->lv.size() >= 2 * (l + 1);
            if (tl) rec_event(ps->lv[2 * l], s);
            if (prof && l == 0) { rec_event(ps->relax0[0], s); ps->relax_timed = true; }
            for (int f = 0; f < fs; ++f, cur ^= 1)
                relax_f<T>(L, (const T *)L.vb, bufs[cur], bufs[cur ^ 1], l == 0 && f == fs - 1 ? x64 : nullptr,
                           l == 0 && f == fs - 1 ? d32 : nullptr, act, any, h.sms, s);
            relax_c<T>(L, (const T *)L.vb, bufs[cur], (T *)L.vx, l == 0 ? x64 : nullptr, l == 0 ? d32 : nullptr,
                       (const T *)L.vx, act, any, h.sms, s);
            if (tl) rec_event(ps->lv[2 * l + 1], s);
            if (prof && l == 0) rec_event(ps->relax0[1], s);
        }
        L.vF = bufs[cur];
    }
    if (NL == 1) {   // single-level hierarchies: x += coarsest solution
        Level &L = h.lev[0];
        launch_pdl(k_fold_coarsest<T>, blocks_for(L.n, BS), BS, s, L.n, (const T *)L.vx, x64, d32, xdd, active,
                   L.rowdir);
        PR_LAUNCH();
    }
}

}  // namespace

void alloc_cycle_vectors(Hier &h) {
    size_t es = h.prm.precision >= 1 ? sizeof(float) : sizeof(double);
    for (auto &L : h.lev) {
        size_t n = (size_t)std::max(L.n, 1);
        L.vb = dmalloc<char>(n * es, h.stream);
        L.vx = dmalloc<char>(n * es, h.stream);
        L.vxn = dmalloc<char>(n * es, h.stream);
        L.vy = dmalloc<char>(n * es, h.stream);
        PR_CUDA(cudaMemsetAsync(L.vx, 0, n * es, h.stream));
        PR_CUDA(cudaMemsetAsync(L.vxn, 0, n * es, h.stream));
        PR_CUDA(cudaMemsetAsync(L.vy, 0, n * es, h.stream));
    }
    int mb = 1;
    for (int d = 0; d < h.ndir; ++d) mb = std::max<int>(mb, (int)blocks_for(h.n0[d], BS));
    if (h.bsr0) mb = std::max<int>(mb, (int)blocks_for(h.hex_n, 32) * h.hex_n * h.hex_n);
    h.maxblk = mb;
    h.partials = dmalloc<double>((size_t)mb * h.ndir, h.stream);
    h.rnorm = dmalloc<double>(h.ndir, h.stream);
    h.rnorm0 = dmalloc<double>(h.ndir, h.stream);
    h.bnorm = dmalloc<double>(h.ndir, h.stream);
    h.active = dmalloc<int>(h.ndir, h.stream);
    set_all_active(h);
    int dev = 0;
    PR_CUDA(cudaGetDevice(&dev));
    PR_CUDA(cudaDeviceGetAttribute(&h.sms, cudaDevAttrMultiProcessorCount, dev));
    autotune_cycle(h);
}

void set_all_active(Hier &h) {
    std::vector<int> ones(h.ndir, 1);
    PR_CUDA(cudaMemcpyAsync(h.active, ones.data(), sizeof(int) * h.ndir, cudaMemcpyHostToDevice, h.stream));
    PR_CUDA(cudaStreamSynchronize(h.stream));   // 'ones' is pageable host memory
}

namespace {
// faces with an upwind neighbour of each level-0 row, split by CF, per matrix
__global__ void k_face_counts(int n, int N, const int8_t *dsign, const int8_t *cf, unsigned long long *out) {
    // out[m][0] = F rows, [1] = C rows, [2] = faces of F rows, [3] = faces of C rows
    __shared__ unsigned long long sh[4];
    int m = blockIdx.y;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (threadIdx.x < 4) sh[threadIdx.x] = 0;
    __syncthreads();
    if (i < N) {
        int e = i >> 3;
        int idx[3] = {e % n, (e / n) % n, e / (n * n)};
        int f = 0;
        for (int d = 0; d < 3; ++d) {
            int sg = dsign[3 * m + d];
            if (sg != 0 && (sg > 0 ? idx[d] > 0 : idx[d] < n - 1)) ++f;
        }
        bool isC = cf[(long long)m * N + i] == CF_C;
        atomicAdd(&sh[isC ? 1 : 0], 1ULL);
        atomicAdd(&sh[isC ? 3 : 2], (unsigned long long)f);
    }
    __syncthreads();
    if (threadIdx.x < 4) atomicAdd(&out[4 * m + threadIdx.x], sh[threadIdx.x]);
}
}  // namespace

namespace {
// per level: [F rows, C rows, entries of F rows, entries of C rows]
__global__ void k_level_counts(int n, const int *rowptr, const int8_t *cf, unsigned long long *out) {
    __shared__ unsigned long long sh[4];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (threadIdx.x < 4) sh[threadIdx.x] = 0;
    __syncthreads();
    if (i < n && cf[i] != CF_COARSEST) {
        bool isC = cf[i] == CF_C;
        atomicAdd(&sh[isC ? 1 : 0], 1ULL);
        atomicAdd(&sh[isC ? 3 : 2], (unsigned long long)(rowptr[i + 1] - rowptr[i]));
    }
    __syncthreads();
    if (threadIdx.x < 4) atomicAdd(&out[threadIdx.x], sh[threadIdx.x]);
}
// level 0 in CSR form, per matrix: [F rows, C rows, entries of F rows, entries of C rows]
// (a warp whose rows all belong to one matrix sums its counts first: one atomic
// per counter and warp instead of one per row)
__global__ void k_level_counts_dir(int n, const int *rowptr, const int8_t *cf, const int *rowdir,
                                   unsigned long long *out) {
    const unsigned FULL = 0xffffffffu;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < n && cf[i] != CF_COARSEST;
    const int d = i < n ? rowdir[i] : -1;
    unsigned long long c[4] = {0, 0, 0, 0};
    if (valid) {
        const bool isC = cf[i] == CF_C;
        c[isC ? 1 : 0] = 1;
        c[isC ? 3 : 2] = (unsigned long long)(rowptr[i + 1] - rowptr[i]);
    }
    const int d0 = __shfl_sync(FULL, d, 0);
    if (__all_sync(FULL, d == d0 || d < 0)) {
        for (int k = 0; k < 4; ++k)
            for (int o = 16; o > 0; o >>= 1) c[k] += __shfl_xor_sync(FULL, c[k], o);
        if ((threadIdx.x & 31) == 0 && d0 >= 0)
            for (int k = 0; k < 4; ++k)
                if (c[k]) atomicAdd(&out[4LL * d0 + k], c[k]);
    } else if (valid) {
        for (int k = 0; k < 4; ++k)
            if (c[k]) atomicAdd(&out[4LL * d + k], c[k]);
    }
}
}  // namespace

void level0_bytes(Hier &h) {
    h.bytes_res0.assign(h.ndir, 0.0);
    h.bytes_relax0.assign(h.ndir, 0.0);
    h.bytes_res32.assign(h.ndir, 0.0);
    h.bytes_relaxc = 0;
    h.bytes_xfer = 0;
    {
        // grid transfers: each restriction row reads its position (row index, entry
        // count), its coarse point's fine row and value, writes its coarse value, and
        // reads its entries (column + value); each prolongation reads the CF flag and P
        // column of every non-coarsest fine row and writes its value (and, for C rows,
        // the copy for the F sweeps).  Gathered values are taken as cached.
        const double sT = h.prm.precision >= 1 ? 4.0 : 8.0;
        for (size_t l = 0; l + 1 < h.lev.size(); ++l) {
            const Level &L = h.lev[l];
            if (L.nc <= 0) continue;
            const double cb = L.sZ.col16 ? 2.0 : 4.0;
            h.bytes_xfer += (double)L.nc * (12 + 2 * sT) + (double)L.nnzZ * (cb + sT);
            h.bytes_xfer += (double)(L.nF + L.nC) * (5 + sT) + (double)L.nC * sT;
        }
    }
    // the iterate the level-0 relaxation folds into: FP64 x or a float pair (8 B
    // read + 8 B written per row), or in the inner correction the FP32 d (4 + 4)
    const double xfold = h.inner ? 8.0 : 16.0;
    cudaStream_t s = h.stream;
    {
        // coarse levels: each F sweep reads, per F row, its split position (row index and
        // entry offset), b, dinv and its input value, writes its output value, and reads
        // its entries (column + value); the C sweep likewise over the C rows.  Gathered
        // neighbour values are taken as cached (the vector is far smaller than L2).
        double sT = h.prm.precision >= 1 ? 4.0 : 8.0;
        unsigned long long *cnt = dmalloc<unsigned long long>(4, s);
        for (size_t l = 1; l + 1 < h.lev.size(); ++l) {
            Level &L = h.lev[l];
            if (L.n == 0) continue;
            PR_CUDA(cudaMemsetAsync(cnt, 0, 4 * sizeof(unsigned long long), s));
            k_level_counts<<<blocks_for(L.n, BS), BS, 0, s>>>(L.n, L.rowptr, L.cf, cnt);
            PR_LAUNCH();
            unsigned long long c[4];
            PR_CUDA(cudaMemcpyAsync(c, cnt, sizeof c, cudaMemcpyDeviceToHost, s));
            PR_CUDA(cudaStreamSynchronize(s));
            // column index: 4 bytes, or 2 in a store with 16-bit offsets
            const double cbF = L.sF.col16 ? 2.0 : 4.0, cbC = L.sC.col16 ? 2.0 : 4.0;
            double fpass = (double)c[0] * (8 + 4 * sT) + (double)c[2] * (cbF + sT);
            double cpass = (double)c[1] * (8 + 4 * sT) + (double)c[3] * (cbC + sT);
            h.bytes_relaxc += h.prm.f_sweeps * fpass + cpass;
        }
        dfree(cnt, s);
        // grid-wide coarsest sweeps: the first reads each row's split position, b and
        // dinv and writes its value; each further one counts as an F sweep
        for (size_t l = 1; l < h.lev.size(); ++l) {
            const Level &L = h.lev[l];
            if (L.sX.nrows <= 0 || h.prm.coarse_sweeps <= 0) continue;
            double nz = 0;
            for (int d = 0; d < h.ndir; ++d)
                if (L.nrows[d] > 0 && L.coarsest[d]) nz += L.nnzdir[d];
            const double nx = L.sX.nrows, cb = L.sX.col16 ? 2.0 : 4.0;
            h.bytes_relaxc += nx * (4 + 3 * sT) + (h.prm.coarse_sweeps - 1) * (nx * (8 + 4 * sT) + nz * (cb + sT));
        }
    }
    if (!h.bsr0) {
        // CSR level 0 (tetrahedra): residual reads every entry (column + FP64 value), b
        // and x, writes r; the relaxation counts as on coarse levels, except that the
        // last F sweep and the C sweep add into x64 (read + write) instead of writing
        Level &L = h.lev[0];
        double sT = h.prm.precision >= 1 ? 4.0 : 8.0;
        unsigned long long *cnt = dmalloc<unsigned long long>(4 * h.ndir, s);
        PR_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * 4 * h.ndir, s));
        k_level_counts_dir<<<blocks_for(std::max(L.n, 1), BS), BS, 0, s>>>(L.n, L.rowptr, L.cf, L.rowdir, cnt);
        PR_LAUNCH();
        std::vector<unsigned long long> c(4 * h.ndir);
        PR_CUDA(cudaMemcpyAsync(c.data(), cnt, sizeof(unsigned long long) * c.size(), cudaMemcpyDeviceToHost, s));
        PR_CUDA(cudaStreamSynchronize(s));
        dfree(cnt, s);
        for (int m = 0; m < h.ndir; ++m) {
            double nF = (double)c[4 * m], nC = (double)c[4 * m + 1], eF = (double)c[4 * m + 2],
                   eC = (double)c[4 * m + 3];
            // outer residual: entries, b and x read, r written (and its r32 copy)
            h.bytes_res0[m] = (eF + eC) * 12 + (nF + nC) * (16 + sT + (h.inner ? 4 : 0));
            double fpass = nF * (8 + 4 * sT) + eF * (4 + sT);
            double cpass = nC * (8 + 3 * sT + xfold) + eC * (4 + sT);
            h.bytes_relax0[m] = h.prm.f_sweeps * fpass + nF * xfold + cpass;
            // inner residual: row pointer, entries (column + FP32 value), r32 and d read, r written
            if (h.inner) h.bytes_res32[m] = (eF + eC) * 8 + (nF + nC) * 16;
        }
        return;
    }
    int N = h.n0[0];
    unsigned long long *cnt = dmalloc<unsigned long long>(4 * h.ndir, s);
    PR_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * 4 * h.ndir, s));
    dim3 grid(blocks_for(N, BS), h.ndir);
    k_face_counts<<<grid, BS, 0, s>>>(h.hex_n, N, h.dsign, h.lev[0].cf, cnt);
    PR_LAUNCH();
    std::vector<unsigned long long> c(4 * h.ndir);
    PR_CUDA(cudaMemcpyAsync(c.data(), cnt, sizeof(unsigned long long) * c.size(), cudaMemcpyDeviceToHost, s));
    PR_CUDA(cudaStreamSynchronize(s));
    dfree(cnt, s);
    double sT = h.prm.precision >= 1 ? 4.0 : 8.0;
    for (int m = 0; m < h.ndir; ++m) {
        double nF = (double)c[4 * m], nC = (double)c[4 * m + 1], fF = (double)c[4 * m + 2], fC = (double)c[4 * m + 3];
        // residual: FP64 face rows (4 values each), b, x read, r written (cycle precision)
        // and, in the inner correction, its r32 copy
        h.bytes_res0[m] = (fF + fC) * 4 * 8 + (nF + nC) * (8 + 8 + sT + (h.inner ? 4 : 0));
        // inner residual: FP32 face rows, r32 and d read, r written
        if (h.inner) h.bytes_res32[m] = (fF + fC) * 4 * 4 + (nF + nC) * 12;
        // each F pass: cf, input and output vector for all rows; A rows and b for F rows
        // C pass: cf, input, x64 (read + write) for all rows; A rows and b for C rows
        if (h.split0) {
            // F sweep: per F row its index, input, b and output, and 4 values per upwind
            // face; the last one also reads and writes x (16 B); C sweep: per C row its
            // index, input, b, x read + write, and its faces' values
            double fpass = fF * 4 * sT + nF * (4 + 3 * sT);
            h.bytes_relax0[m] = h.prm.f_sweeps * fpass + nF * xfold + fC * 4 * sT + nC * (4 + 2 * sT + xfold);
        } else {
            double fpass = fF * 4 * sT + (nF + nC) * (1 + 2 * sT) + nF * sT;
            h.bytes_relax0[m] = h.prm.f_sweeps * fpass + fC * 4 * sT + (nF + nC) * (1 + sT + 16) + nC * sT;
        }
    }
}

void prof_enable(Hier &h) {
    if (h.prof) return;
    for (auto &e : h.ev) PR_CUDA(cudaEventCreate(&e));
    h.slots.resize(h.inner ? INNER_SLOTS : 1);
    for (auto &ps : h.slots) {
        for (auto &e : ps.relax0) PR_CUDA(cudaEventCreate(&e));
        for (auto &e : ps.res32) PR_CUDA(cudaEventCreate(&e));
        ps.lv.assign(2 * h.lev.size(), nullptr);
        for (auto &e : ps.lv) PR_CUDA(cudaEventCreate(&e));
        ps.lvx.assign(2 * h.lev.size(), nullptr);
        for (auto &e : ps.lvx) PR_CUDA(cudaEventCreate(&e));
        ps.lvt.assign(4 * h.lev.size(), nullptr);
        for (auto &e : ps.lvt) PR_CUDA(cudaEventCreate(&e));
    }
    h.prof = true;
}

namespace {
// outer residual kernels: r = b - A0 x into lev[0].vb (and r2, if given), the
// per-matrix partial sums of squares into h.partials
void residual0_launch(Hier &h, const double *b, const double *x, const int *act, float *r2, bool zero_x = false) {
    cudaStream_t s = h.stream;
    Level &L = h.lev[0];
    dim3 grid(h.maxblk, h.ndir);
    bool f32 = h.prm.precision >= 1;
    if (h.bsr0 && h.dd) {
        int N = h.n0[0];
        dim3 g3(blocks_for(h.hex_n, 32), h.hex_n * h.hex_n, h.ndir);
        launch_pdl(k_res0_bsr_dd, g3, BS, s, h.hex_n, N, h.dsign, h.bsr_dd, h.b_dd, h.x_dd, (float *)L.vb, r2,
                   h.partials, h.maxblk, act);
    } else if (h.bsr0) {
        int N = h.n0[0];
        dim3 g3(blocks_for(h.hex_n, 32), h.hex_n * h.hex_n, h.ndir);
        if (f32)
            launch_pdl(k_res0_bsr<float>, g3, BS, s, h.hex_n, N, h.dsign, h.bsr64, b, x, (float *)L.vb, r2,
                       h.partials, h.maxblk, act, zero_x ? 1 : 0);
        else
            launch_pdl(k_res0_bsr<double>, g3, BS, s, h.hex_n, N, h.dsign, h.bsr64, b, x, (double *)L.vb,
                       (float *)nullptr, h.partials, h.maxblk, act, zero_x ? 1 : 0);
    } else {
        if (f32)
            launch_pdl(k_res0_csr<float>, grid, BS, s, h.d_row00, h.d_n0, L.rowptr, L.col, L.val, b, x, (float *)L.vb,
                       r2, h.partials, h.maxblk, act, zero_x ? 1 : 0);
        else
            launch_pdl(k_res0_csr<double>, grid, BS, s, h.d_row00, h.d_n0, L.rowptr, L.col, L.val, b, x,
                       (double *)L.vb, (float *)nullptr, h.partials, h.maxblk, act, zero_x ? 1 : 0);
    }
    PR_LAUNCH();
}
}  // namespace

void residual0(Hier &h, const double *b, const double *x, double tol, bool update_active, bool zero_x) {
    cudaStream_t s = h.stream;
    // every block of an active matrix writes its partial; inactive matrices' partials
    // are not read
    int *act = update_active ? h.active : nullptr;
    const bool tm = h.timed && !zero_x;   // timings cover the residuals that read the operator
    if (tm) rec_event(h.ev[0], s);
    residual0_launch(h, b, x, act, nullptr, zero_x && !h.dd);
    if (tm) rec_event(h.ev[1], s);
    launch_pdl(k_norm_final, blocks_for(32LL * h.ndir, 128), 128, s, h.ndir, h.partials, h.maxblk, h.rnorm, h.bnorm, tol,
                                                                 act);
    PR_LAUNCH();
}

void norms0(Hier &h, const double *v, double *out) {
    cudaStream_t s = h.stream;
    PR_CUDA(cudaMemsetAsync(h.partials, 0, sizeof(double) * h.maxblk * h.ndir, s));
    dim3 grid(h.maxblk, h.ndir);
    if (h.prm.precision >= 1) k_sumsq_rows<true><<<grid, BS, 0, s>>>(h.d_row00, h.d_n0, v, h.partials, h.maxblk);
    else k_sumsq_rows<false><<<grid, BS, 0, s>>>(h.d_row00, h.d_n0, v, h.partials, h.maxblk);
    PR_LAUNCH();
    k_norm_final<<<blocks_for(32LL * h.ndir, 128), 128, 0, s>>>(h.ndir, h.partials, h.maxblk, out, nullptr, 0.0,
                                                                 nullptr);
    PR_LAUNCH();
}

void dd_enable(Hier &h) {
    if (!h.bsr0 || h.prm.precision != 2 || !h.bsr64) return;
    cudaStream_t s = h.stream;
    const long long nv = (long long)h.ndir * (h.n0[0] / 8) * 96;
    h.bsr_dd = dmalloc<float2>(nv, s);
    k_dd_split<<<blocks_for(nv, BS), BS, 0, s>>>(nv, h.bsr64, h.bsr_dd);
    PR_LAUNCH();
    dfree(h.bsr64, s);
    h.bsr64 = nullptr;
    const long long nr = (long long)h.ndir * h.n0[0];
    h.b_dd = dmalloc<float2>(nr, s);
    h.x_dd = dmalloc<float2>(nr, s);
    h.dd = true;
}

void split0_enable(Hier &h) {
    if (!h.bsr0 || h.prm.precision < 1 || !h.bsr32) return;
    Level &L = h.lev[0];
    if (!L.srow) return;
    cudaStream_t s = h.stream;
    h.v0 = dmalloc<float4>(3LL * std::max(L.n, 1), s);
    k_split0_copy<<<blocks_for(L.n, BS), BS, 0, s>>>(L.n, h.n0[0], L.srow, h.bsr32, h.v0);
    PR_LAUNCH();
    if (!h.inner) {   // the inner correction's FP32 residual reads the element-ordered copy
        dfree(h.bsr32, s);
        h.bsr32 = nullptr;
    }
    h.split0 = true;
}

void dd_load(Hier &h, const double *b, const double *x) {
    const long long nr = (long long)h.ndir * h.n0[0];
    k_dd_split<<<blocks_for(nr, BS), BS, 0, h.stream>>>(nr, b, h.b_dd);
    PR_LAUNCH();
    k_dd_split<<<blocks_for(nr, BS), BS, 0, h.stream>>>(nr, x, h.x_dd);
    PR_LAUNCH();
}

void dd_store(Hier &h, double *x) {
    const long long nr = (long long)h.ndir * h.n0[0];
    k_dd_join<<<blocks_for(nr, BS), BS, 0, h.stream>>>(nr, h.x_dd, x);
    PR_LAUNCH();
}

// ---- autotuner ---------------------------------------------------------------------
// For every SELL store (F sweep, C sweep, restriction on every level) the lanes per
// row G in {1, 2, 4, 8} are timed with CUDA events on the store itself (one warm-up
// and three timed launches each, on the zeroed cycle vectors, before the hierarchy's
// first cycle) and the fastest is kept.  Choices are cached for the process by
// (kernel, precision, positions, stored entries), so rebuilding a hierarchy of the
// same shape (the next batch, the next source iteration) reuses them.
namespace {
std::mutex g_tune_mutex;
std::map<std::tuple<int, int, int, long long>, int> g_tune;

template <class T, int MODE>
void tune_store(Sell &S, const SellJob<T> &j, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1) {
    if (S.nrows <= 0) return;
    const auto key = std::make_tuple(MODE, (int)sizeof(T), S.npos, S.nnz);
    // held while tuning: hierarchies set up at the same time on other threads (the
    // concurrent direction groups) with a store of the same key wait for this choice
    // instead of timing their own, so equal stores of one process sum rows alike
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) { S.G = it->second; return; }
    int best = 1;
    float tbest = 0;
    for (int G = 1; G <= 8; G *= 2) {
        launch_sell_g<T, MODE>(S, j, G, s);
        PR_CUDA(cudaEventRecord(e0, s));
        for (int r = 0; r < 3; ++r) launch_sell_g<T, MODE>(S, j, G, s);
        PR_CUDA(cudaEventRecord(e1, s));
        PR_CUDA(cudaEventSynchronize(e1));
        float ms = 0;
        PR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (G == 1 || ms < tbest) { tbest = ms; best = G; }
    }
    S.G = best;
    g_tune[key] = best;
}

template <class T>
void autotune_t(Hier &h) {
    cudaStream_t s = h.stream;
    cudaEvent_t e0, e1;
    PR_CUDA(cudaEventCreate(&e0));
    PR_CUDA(cudaEventCreate(&e1));
    struct Ev {
        cudaEvent_t a, b;
        ~Ev() { cudaEventDestroy(a); cudaEventDestroy(b); }
    } ev{e0, e1};
    const int NL = (int)h.lev.size();
    for (int l = 0; l < NL; ++l) {
        Level &L = h.lev[l];
        SellJob<T> j{};
        j.in = (const T *)L.vy;
        j.dinv = lv_dinv<T>(L);
        j.b = (const T *)L.vb;
        j.out = (T *)L.vxn;
        j.rowdir = L.rowdir;
        tune_store<T, SM_F>(L.sF, j, s, e0, e1);
        tune_store<T, SM_C>(L.sC, j, s, e0, e1);
        tune_store<T, SM_F>(L.sX, j, s, e0, e1);
        if (l + 1 < NL && L.sZ.nrows > 0) {
            SellJob<T> r{};
            r.in = (const T *)L.vb;
            r.out = (T *)h.lev[l + 1].vb;
            r.cpts = L.cpts;
            tune_store<T, SM_RESTRICT>(L.sZ, r, s, e0, e1);
        }
    }
    // the tuning launches wrote only the zeroed work vectors: clear them again
    size_t es = sizeof(T);
    for (auto &L : h.lev) {
        size_t n = (size_t)std::max(L.n, 1);
        PR_CUDA(cudaMemsetAsync(L.vb, 0, n * es, s));
        PR_CUDA(cudaMemsetAsync(L.vxn, 0, n * es, s));
    }
    PR_CUDA(cudaStreamSynchronize(s));
}
}  // namespace

void autotune_cycle(Hier &h) {
    if (h.prm.precision >= 1) autotune_t<float>(h);
    else autotune_t<double>(h);
}

void inner_enable(Hier &h) {
    if (h.prm.precision < 1 || h.inner) return;
    cudaStream_t s = h.stream;
    Level &L = h.lev[0];
    const size_t rows = (size_t)std::max(L.n, 1);
    h.r32 = dmalloc<float>(rows, s);
    h.d32 = dmalloc<float>(rows, s);
    PR_CUDA(cudaMemsetAsync(h.d32, 0, rows * sizeof(float), s));
    h.iactive = dmalloc<int>(h.ndir, s);
    h.icount = dmalloc<int>(h.ndir, s);
    h.iany = dmalloc<int>(1, s);
    PR_CUDA(cudaMemsetAsync(h.iany, 0, sizeof(int), s));
    h.iticket = dmalloc<unsigned>(1, s);
    PR_CUDA(cudaMemsetAsync(h.iticket, 0, sizeof(unsigned), s));
    h.ithr = dmalloc<double>(h.ndir, s);
    h.inorm = dmalloc<double>(h.ndir, s);
    PR_CUDA(cudaMemsetAsync(h.iactive, 0, sizeof(int) * h.ndir, s));
    PR_CUDA(cudaMemsetAsync(h.icount, 0, sizeof(int) * h.ndir, s));
    if (h.bsr0) {
        PR_REQUIRE(h.bsr32, PAIR_ERR_DEVICE, "inner correction: no FP32 block form");
    } else {
        h.val32 = dmalloc<float>((size_t)std::max<long long>(L.nnz, 1), s);
        k_to_f32<<<blocks_for(std::max<long long>(L.nnz, 1), BS), BS, 0, s>>>(L.nnz, L.val, h.val32);
        PR_LAUNCH();
    }
    h.inner = true;
}

void residual_outer(Hier &h, const double *b, const double *x, double tol, bool zero_x) {
    cudaStream_t s = h.stream;
    const bool tm = h.timed && !zero_x;   // timings cover the residuals that read the operator
    if (tm) rec_event(h.ev[0], s);
    residual0_launch(h, b, x, h.active, h.r32, zero_x && !h.dd);
    if (tm) rec_event(h.ev[1], s);
    launch_pdl(k_norm_outer, h.ndir, NORM_BS, s, h.ndir, (const double *)h.partials, h.maxblk, h.rnorm,
               (const double *)h.bnorm, tol, h.active, h.iactive, h.ithr, h.iany, h.iticket);
    PR_LAUNCH();
}

void inner_cycle(Hier &h, ProfSlot *ps) {
    cudaStream_t s = h.stream;
    vcycle_t<float>(h, nullptr, h.d32, h.iactive, ps);
    const bool prof = h.timed && ps;
    if (ps) ps->res_timed = false;
    if (prof) { rec_event(ps->res32[0], s); ps->res_timed = true; }
    Level &L = h.lev[0];
    if (h.bsr0) {
        dim3 g3(blocks_for(h.hex_n, 32), h.hex_n * h.hex_n, h.ndir);
        launch_pdl(k_res32_bsr, g3, BS, s, h.hex_n, h.n0[0], h.dsign, (const float *)h.bsr32, (const float *)h.r32,
                   (const float *)h.d32, (float *)L.vb, h.partials, h.maxblk, (const int *)h.iactive);
    } else {
        dim3 grid(h.maxblk, h.ndir);
        launch_pdl(k_res32_csr, grid, BS, s, (const int *)h.d_row00, (const int *)h.d_n0, (const int *)L.rowptr,
                   (const int *)L.col, (const float *)h.val32, (const float *)h.r32, (const float *)h.d32,
                   (float *)L.vb, h.partials, h.maxblk, (const int *)h.iactive);
    }
    PR_LAUNCH();
    if (prof) rec_event(ps->res32[1], s);
    launch_pdl(k_norm_inner, h.ndir, NORM_BS, s, h.ndir, (const double *)h.partials, h.maxblk, h.inorm,
               (const double *)h.ithr, h.iactive, h.icount, h.iany, h.iticket);
    PR_LAUNCH();
}

void fold_delta(Hier &h, double *x) {
    dim3 grid(h.maxblk, h.ndir);
    launch_pdl(k_fold_delta, grid, BS, h.stream, (const int *)h.d_row00, (const int *)h.d_n0, h.d32, x,
               h.dd ? h.x_dd : (float2 *)nullptr, (const int *)h.active);
    PR_LAUNCH();
}

void vcycle_correct(Hier &h, double *x, ProfSlot *ps) {
    if (h.prm.precision >= 1) vcycle_t<float>(h, x, nullptr, h.active, ps);
    else vcycle_t<double>(h, x, nullptr, h.active, ps);
}

}  // namespace pr
