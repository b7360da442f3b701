// AIR setup on the GPU (Sec. 1.2; Sec. 4.1.1 Eq. soc; Sec. 4.1.2 filtering).
//
// A hierarchy holds a batch of independent matrices; every level of every
// matrix is processed by one launch per step.  Compiled with --fmad=false and
// written so that each floating-point result is formed by the same operations
// in the same order as the plain definitions below (fused multiply-adds only
// where fma() is written), hence reproducible bit for bit:
//   strength   S_i = {j != i : |a_ij| >= theta * max_{k != i} |a_ik|}, empty if the max is 0
//   PMIS       key_i = (lambda_i, h_i, i), lambda_i = #{k : i in S_k},
//              h_i = top 32 bits of SplitMix64 at state seed ^ (level << 40) ^ i (local i);
//              lambda_i = 0 -> F; rounds: undecided local key maxima over S + S^T -> C,
//              undecided rows depending strongly on a new C -> F
//   P          one-point: F row -> strongest C neighbour in S_i (first maximum), weight 1
//   lAIR       C row i, pattern R_i = strong (eps_R) F neighbours (distance 1, or 2 via F
//              points), A[R_i,R_i]^T z = -A[i,R_i]^T by LU with partial pivoting (first max
//              pivot, full row swaps, column-oriented substitutions); optional phi_R filter
//   RAP        (AP)[k,c] = sum over l ascending (pmap(l) = c) of a_kl, starting from 0.0;
//              (RAP)[i,c] = sum over the R row in ascending column order (identity at
//              its place) of R_ik (AP)[k,c], starting from 0.0, one fma per term; every
//              structural product kept; optional phi_A filter of off-diagonal entries
//   LU         multipliers a_rk * (1 / a_kk), updates fma(-l, a_kc, a_rc), substitutions
//              by columns with fma, y_k * (1 / u_kk)
#include <algorithm>
#include <cstdio>

#include "common.cuh"

namespace pr {

namespace {

constexpr int8_t ST_U = -1, ST_F = 0, ST_C = 1;

__device__ __forceinline__ uint64_t splitmix_first(uint64_t state) {
    uint64_t z = state + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double lookup(const int *rowptr, const int *col, const double *val, int i, int j) {
    int lo = rowptr[i], hi = rowptr[i + 1] - 1;
    while (lo <= hi) {
        int m = (lo + hi) >> 1;
        int c = col[m];
        if (c == j) return val[m];
        if (c < j) lo = m + 1; else hi = m - 1;
    }
    return 0.0;
}

__global__ void k_dinv(int n, const int *rowptr, const int *col, const double *val, double *dinv, float *dinv32) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double d = lookup(rowptr, col, val, i, i);
    double r = (d != 0.0) ? 1.0 / d : 0.0;
    dinv[i] = r;
    if (dinv32) dinv32[i] = (float)r;
}

// bit 0: S (theta), bit 1: S^R (eps_R)
__global__ void k_strength(int n, const int *rowptr, const int *col, const double *val, const int *rowdir,
                           const char *dwork, double theta, double epsR, uint8_t *S) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int p0 = rowptr[i], p1 = rowptr[i + 1];
    if (!dwork[rowdir[i]]) {
        for (int p = p0; p < p1; ++p) S[p] = 0;
        return;
    }
    double m = 0.0;
    for (int p = p0; p < p1; ++p)
        if (col[p] != i) { double v = fabs(val[p]); if (v > m) m = v; }
    double t1 = theta * m, t2 = epsR * m;
    for (int p = p0; p < p1; ++p) {
        uint8_t s = 0;
        if (col[p] != i && m > 0.0) {
            double a = fabs(val[p]);
            if (a >= t1) s |= 1;
            if (a >= t2) s |= 2;
        }
        S[p] = s;
    }
}

__global__ void k_lambda(int n, const int *rowptr, const int *col, const uint8_t *S, unsigned *lam) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p)
        if (S[p] & 1) atomicAdd(&lam[col[p]], 1u);
}

__global__ void k_pmis_init(int n, const int *rowdir, const char *dwork, const int *row0, const unsigned *lam,
                            int level, unsigned long long seed, uint64_t *key, int8_t *state, int *undecided) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int d = rowdir[i];
    if (!dwork[d]) { state[i] = ST_F; key[i] = 0; return; }
    uint64_t li = (uint64_t)(i - row0[d]);
    uint32_t hh = (uint32_t)(splitmix_first(seed ^ ((uint64_t)level << 40) ^ li) >> 32);
    key[i] = ((uint64_t)lam[i] << 32) | hh;
    int8_t s = lam[i] == 0 ? ST_F : ST_U;
    state[i] = s;
    if (s == ST_U) atomicAdd(undecided, 1);
}

__device__ __forceinline__ bool key_gt(uint64_t kj, int j, uint64_t ki, int i) {
    return kj > ki || (kj == ki && j > i);
}

__global__ void k_pmis_mark(int n, const int *rowptr, const int *col, const uint8_t *S, const uint64_t *key,
                            const int8_t *state, int *notmax, int round) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || state[i] != ST_U) return;
    uint64_t ki = key[i];
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
        if (!(S[p] & 1)) continue;
        int j = col[p];
        if (state[j] != ST_U) continue;
        if (key_gt(key[j], j, ki, i)) notmax[i] = round;
        else notmax[j] = round;
    }
}

__global__ void k_pmis_update(int n, const int *rowptr, const int *col, const uint8_t *S, const int8_t *state,
                              int8_t *next, const int *notmax, int round, int *undecided) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int8_t s = state[i];
    if (s != ST_U) { next[i] = s; return; }
    if (notmax[i] != round) { next[i] = ST_C; return; }
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
        if (!(S[p] & 1)) continue;
        int j = col[p];
        if (state[j] == ST_U && notmax[j] != round) { next[i] = ST_F; return; }
    }
    next[i] = ST_U;
    atomicAdd(undecided, 1);
}

// per-matrix sums: one atomic per warp when its rows share a matrix (the usual case)
template <class T>
__device__ __forceinline__ void add_by_dir(T *out, int d, T v, bool valid) {
    unsigned act = __ballot_sync(0xffffffffu, valid);
    if (!act) return;
    int d0 = __shfl_sync(0xffffffffu, d, __ffs(act) - 1);
    bool same = __all_sync(0xffffffffu, !valid || d == d0);
    if (same) {
        T tot = valid ? v : T(0);
        for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
        if ((threadIdx.x & 31) == __ffs(act) - 1 && tot) atomicAdd(&out[d0], tot);
    } else if (valid && v) {
        atomicAdd(&out[d], v);
    }
}

__global__ void k_count_c(int n, const int *rowdir, const int8_t *state, int *ncdir) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool valid = i < n;
    int d = valid ? rowdir[i] : 0;
    add_by_dir<int>(ncdir, d, (valid && state[i] == ST_C) ? 1 : 0, valid);
}

__global__ void k_cf_final(int n, const int *rowdir, const char *cont, const int8_t *state, int8_t *cf, int *isC) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool c = cont[rowdir[i]];
    cf[i] = c ? (state[i] == ST_C ? CF_C : CF_F) : CF_COARSEST;
    isC[i] = (c && state[i] == ST_C) ? 1 : 0;
}

__global__ void k_cpts(int n, const int8_t *cf, const int *cidx, int *cpts) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (cf[i] == CF_C) cpts[cidx[i]] = i;
}

__global__ void k_pmap(int n, const int *rowptr, const int *col, const double *val, const uint8_t *S,
                       const int8_t *cf, const int *cidx, int *pmap) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int8_t c = cf[i];
    if (c == CF_COARSEST) { pmap[i] = -1; return; }
    if (c == CF_C) { pmap[i] = cidx[i]; return; }
    int best = -1;
    double bv = -1.0;
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
        int j = col[p];
        if ((S[p] & 1) && cf[j] == CF_C) {
            double v = fabs(val[p]);
            if (v > bv) { bv = v; best = j; }
        }
    }
    pmap[i] = best >= 0 ? cidx[best] : -1;
}

// ---- lAIR ------------------------------------------------------------------
__global__ void k_lair_ncand(int nc, const int *cpts, const int *rowptr, const int *col, const uint8_t *S,
                             const int8_t *cf, int distance, int *ncand) {
    int ic = blockIdx.x * blockDim.x + threadIdx.x;
    if (ic >= nc) return;
    int i = cpts[ic];
    int c = 0;
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
        int j = col[p];
        if ((S[p] & 2) && cf[j] == CF_F) {
            ++c;
            if (distance >= 2)
                for (int q = rowptr[j]; q < rowptr[j + 1]; ++q)
                    if ((S[q] & 2) && cf[col[q]] == CF_F) ++c;
        }
    }
    ncand[ic] = c;
}

__global__ void k_lair_pattern(int nc, const int *cpts, const int *rowptr, const int *col, const uint8_t *S,
                               const int8_t *cf, int distance, const int *candptr, int *cand, int *npat) {
    int ic = blockIdx.x * blockDim.x + threadIdx.x;
    if (ic >= nc) return;
    int i = cpts[ic];
    int *c = cand + candptr[ic];
    int m = 0;
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
        int j = col[p];
        if ((S[p] & 2) && cf[j] == CF_F) c[m++] = j;
    }
    if (distance >= 2) {
        int m1 = m;
        for (int t = 0; t < m1; ++t) {
            int j = c[t];
            for (int q = rowptr[j]; q < rowptr[j + 1]; ++q)
                if ((S[q] & 2) && cf[col[q]] == CF_F) c[m++] = col[q];
        }
        for (int a = 1; a < m; ++a) {   // insertion sort, then unique
            int v = c[a], b = a;
            while (b > 0 && c[b - 1] > v) { c[b] = c[b - 1]; --b; }
            c[b] = v;
        }
        int u = 0;
        for (int a = 0; a < m; ++a)
            if (u == 0 || c[u - 1] != c[a]) c[u++] = c[a];
        m = u;
    }
    npat[ic] = m;
}

// lAIR systems binned by size: a thread per system up to 8 unknowns (bins of 4, 6
// and 8, whose shared workspaces keep more systems in flight per SM the smaller
// they are), 8 lanes per system up to 16, then a warp per system with a
// shared-memory workspace sized to the bin, global workspaces beyond 64
constexpr int LAIR_CLASSES = 10;
constexpr int LAIR_BIG = LAIR_CLASSES - 1;
__device__ __forceinline__ int lair_class(int np) {
    return np <= 4 ? 0 : np <= 6 ? 1 : np <= 8 ? 2 : np <= 12 ? 3 : np <= 16 ? 4 : np <= 24 ? 5 : np <= 32 ? 6
         : np <= 48 ? 7 : np <= 64 ? 8 : 9;
}



// Warp per C row.  Shared memory per warp: M (nmax^2 doubles), y (nmax
// doubles), pattern (nmax ints), pivots (nmax ints).
__device__ __forceinline__ int pat_find(const int *pat, int np, int k) {
    int lo = 0, hi = np - 1;
    while (lo <= hi) {
        int m = (lo + hi) >> 1;
        int v = pat[m];
        if (v == k) return m;
        if (v < k) lo = m + 1; else hi = m - 1;
    }
    return -1;
}

// ---- nAIR of degree 1 (Neumann series cut after the linear term) -----------
// Thread per C point, on the distance-2 pattern (sorted, from k_lair_pattern):
//   t_k = a_ik for strong F neighbours k of i (else 0); for every strong F
//   neighbour j of i (ascending) and every strong F neighbour k != j of j
//   (ascending): t_k = fma(a_ij, n_jk, t_k), n_jk = -(a_jk * (1/a_jj));
//   z_k = -(t_k * (1/a_kk)), i.e. Z_i = -A_CF^s[i,:] (I + N) D^{-1} with
//   N = I - D^{-1} A_FF^s.  A zero diagonal on the way empties the row (counted
//   as singular).  The values are accumulated in the row's slots of zval and the
//   phi_R filter compacts them in place.
__global__ void k_nair(int nc, const int *cpts, const int *rowptr, const int *col, const double *val,
                       const uint8_t *S, const int8_t *cf, const double *dinv, const int *candptr, const int *cand,
                       const int *npat, const int *zrowptr, int *zcol, double *zval, int *keep, int *nsing_dir,
                       const int *rowdir, double phi_R) {
    int ic = blockIdx.x * blockDim.x + threadIdx.x;
    if (ic >= nc) return;
    const int i = cpts[ic];
    const int np = npat[ic];
    const int *pat = cand + candptr[ic];
    const int base = zrowptr[ic];
    double *t = zval + base;
    for (int e = 0; e < np; ++e) t[e] = 0.0;
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
        int k = col[p];
        if ((S[p] & 2) && cf[k] == CF_F) t[pat_find(pat, np, k)] = val[p];
    }
    bool singular = false;
    for (int p = rowptr[i]; p < rowptr[i + 1] && !singular; ++p) {
        int j = col[p];
        if (!((S[p] & 2) && cf[j] == CF_F)) continue;
        const double aij = val[p], rj = dinv[j];
        if (rj == 0.0) { singular = true; break; }
        for (int q = rowptr[j]; q < rowptr[j + 1]; ++q) {
            int k = col[q];
            if (k == j || !((S[q] & 2) && cf[k] == CF_F)) continue;
            const double njk = -(val[q] * rj);
            const int e = pat_find(pat, np, k);
            t[e] = fma(aij, njk, t[e]);
        }
    }
    for (int e = 0; e < np && !singular; ++e)
        if (dinv[pat[e]] == 0.0) singular = true;
    int kept = 0;
    if (singular) {
        atomicAdd(&nsing_dir[rowdir[i]], 1);
    } else {
        long long zmb = 0;
        for (int e = 0; e < np; ++e) {
            t[e] = -(t[e] * dinv[pat[e]]);
            zmb = max(zmb, absbits(t[e]));
        }
        const double thr = phi_R * __longlong_as_double(zmb);
        for (int e = 0; e < np; ++e) {
            const double z = t[e];
            if (phi_R > 0.0 && fabs(z) < thr) continue;
            zcol[base + kept] = pat[e];
            zval[base + kept] = z;
            ++kept;
        }
    }
    keep[ic] = kept;
}


// 1 / p for a pivot p.  A pivot of magnitude 1 (the unit diagonal of the
// block-scaled level 0, which most eliminations leave untouched) is its own
// reciprocal, exactly, so it takes no division: an FP64 division occupies the FP64
// pipe for a whole warp instruction however few lanes take part, and one per pivot
// was most of the FP64 work left once zero-multiplier rows are skipped.
__device__ __forceinline__ double pivot_recip(double p) {
    const long long mag = __double_as_longlong(p) & 0x7fffffffffffffffLL;   // |p| == 1, integer test
    return mag == 0x3ff0000000000000LL ? p : 1.0 / p;
}

// The FP64 pipe takes a whole warp instruction for any number of active lanes, so
// the O(n^2) passes of the local solves keep their zero tests and signed zeros on
// the integer pipe.
__device__ __forceinline__ bool is_zero_bits(double x) { return (__double_as_longlong(x) & 0x7fffffffffffffffLL) == 0; }
// a * r for a zero a and a finite nonzero r: the zero with the product's sign
__device__ __forceinline__ double zero_times(double a, double r) {
    return __longlong_as_double((__double_as_longlong(a) ^ __double_as_longlong(r)) & (long long)0x8000000000000000ULL);
}
// y * r for a reciprocal r of magnitude 1 (unit pivot): exact sign flip or y itself
__device__ __forceinline__ double times_recip(double y, double r) {
    const long long rb = __double_as_longlong(r);
    if ((rb & 0x7fffffffffffffffLL) == 0x3ff0000000000000LL)
        return __longlong_as_double(__double_as_longlong(y) ^ (rb & (long long)0x8000000000000000ULL));
    return y * r;
}

// Thread per C row of the worklist for systems of size <= NM: every lane of a
// warp works on its own system, so each FP64 instruction carries 32 useful
// operations.  Workspaces live in shared memory interleaved by thread
// (element e of thread t at [e * T + t]), which keeps accesses conflict-free.
template <int NM>
__global__ void __launch_bounds__(64) k_lair_solve_thread(int nwork, const int *worklist, const int *cpts,
                                                          const int *rowptr, const int *col, const double *val,
                                                          const int *candptr, const int *cand, const int *npat,
                                                          const int *zrowptr, int *zcol, double *zval, int *keep,
                                                          int *nsing_dir, const int *rowdir, double phi_R) {
    constexpr int T = 64;
    extern __shared__ double sm3[];
    const int t = threadIdx.x;
    double *Ms = sm3;                   // NM*NM
    double *ys = sm3 + NM * NM * T;     // NM
    double *rs = ys + NM * T;           // NM
    int *ps = (int *)(rs + NM * T);     // NM pattern, NM pivots
#define MM(e) Ms[(e) * T + t]
#define YY(e) ys[(e) * T + t]
#define RR(e) rs[(e) * T + t]
#define PAT(e) ps[(e) * T + t]
#define PIV(e) ps[(NM + (e)) * T + t]
    int w = blockIdx.x * T + t;
    if (w >= nwork) return;
    int ic = worklist[w];
    int i = cpts[ic];
    int np = npat[ic];
    if (np > NM) { keep[ic] = 0; return; }   // excluded by the size bins
    const int *cp = cand + candptr[ic];
    for (int e = 0; e < np; ++e) { PAT(e) = cp[e]; YY(e) = -0.0; }
    for (int e = 0; e < np * np; ++e) MM(e) = 0.0;
    for (int c = 0; c < np; ++c) {
        const int j = PAT(c), p1 = rowptr[j + 1];
        for (int p = rowptr[j]; p < p1; p += 4) {   // four entries' loads before their lookups
            int kk[4];
            double vv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                kk[u] = p + u < p1 ? col[p + u] : -1;
                vv[u] = p + u < p1 ? val[p + u] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int k = kk[u];
                if (k < 0) continue;
                int lo = 0, hi = np - 1, r = -1;
                while (lo <= hi) {
                    int m = (lo + hi) >> 1;
                    int v = PAT(m);
                    if (v == k) { r = m; break; }
                    if (v < k) lo = m + 1; else hi = m - 1;
                }
                if (r >= 0) MM(r * np + c) = vv[u];
            }
        }
    }
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
        int k = col[p], lo = 0, hi = np - 1, r = -1;
        while (lo <= hi) {
            int m = (lo + hi) >> 1;
            int v = PAT(m);
            if (v == k) { r = m; break; }
            if (v < k) lo = m + 1; else hi = m - 1;
        }
        if (r >= 0) YY(r) = -val[p];
    }
    long long mxb = 0;
    for (int e = 0; e < np * np; ++e) mxb = max(mxb, absbits(MM(e)));
    long long tinyb = absbits(1e-14 * __longlong_as_double(mxb));
    bool singular = false;
    for (int k = 0; k < np; ++k) {
        int p = k;
        long long pv = absbits(MM(k * np + k));
        for (int r = k + 1; r < np; ++r) {
            long long v = absbits(MM(r * np + k));
            if (v > pv) { pv = v; p = r; }
        }
        PIV(k) = p;
        if (!(pv > tinyb)) { singular = true; break; }
        if (p != k)
            for (int c = 0; c < np; ++c) { double tt = MM(k * np + c); MM(k * np + c) = MM(p * np + c); MM(p * np + c) = tt; }
        double rd = pivot_recip(MM(k * np + k));
        RR(k) = rd;
        for (int r = k + 1; r < np; ++r) {
            const double a = MM(r * np + k);
            if (is_zero_bits(a)) {   // adds exact zeros: skipped, as in the reference LU
                MM(r * np + k) = zero_times(a, rd);
                continue;
            }
            const double l = a * rd;
            MM(r * np + k) = l;
            if (is_zero_bits(l)) continue;   // (an underflowed multiplier likewise)
            for (int c = k + 1; c < np; ++c) MM(r * np + c) = fma(-l, MM(k * np + c), MM(r * np + c));
        }
    }
    int kept = 0;
    if (singular) {
        atomicAdd(&nsing_dir[rowdir[i]], 1);
    } else if (np > 0) {
        for (int k = 0; k < np; ++k) {
            int p = PIV(k);
            if (p != k) { double tt = YY(k); YY(k) = YY(p); YY(p) = tt; }
        }
        for (int k = 0; k < np; ++k) {
            double yk = YY(k);
            for (int r = k + 1; r < np; ++r) YY(r) = fma(-MM(r * np + k), yk, YY(r));
        }
        for (int k = np - 1; k >= 0; --k) {
            double yk = times_recip(YY(k), RR(k));
            YY(k) = yk;
            for (int r = 0; r < k; ++r) YY(r) = fma(-MM(r * np + k), yk, YY(r));
        }
        long long zmb = 0;
        for (int e = 0; e < np; ++e) zmb = max(zmb, absbits(YY(e)));
        double thr = phi_R * __longlong_as_double(zmb);
        int base = zrowptr[ic];
        for (int e = 0; e < np; ++e) {
            double z = YY(e);
            if (phi_R > 0.0 && fabs(z) < thr) continue;
            zcol[base + kept] = PAT(e);
            zval[base + kept] = z;
            ++kept;
        }
    }
    keep[ic] = kept;
#undef MM
#undef YY
#undef RR
#undef PAT
#undef PIV
}

// G lanes per C row of the worklist (32/G systems per warp).  Shared-memory
// mode (gbuf == null): systems of size <= nmax, workspace nmax^2 + 2 nmax
// doubles per group.  Global mode: workspace at gbuf + goff[w].
template <int G>
__global__ void k_lair_solve(int nwork, const int *worklist, const int *cpts, const int *rowptr, const int *col,
                             const double *val, const int *candptr, const int *cand, const int *npat,
                             const int *zrowptr, int *zcol, double *zval, int *keep, int *nsing_dir,
                             const int *rowdir, double phi_R, int nmax, const long long *goff, double *gbuf) {
    extern __shared__ double smem[];
    const unsigned FULL = 0xffffffffu;
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int g = lane % G, q = lane / G;
    int wpb = blockDim.x >> 5;
    constexpr int SPW = 32 / G;   // systems per warp
    const unsigned gmask = (G == 32) ? FULL : (((1u << (G & 31)) - 1u) << (q * G));   // this group's lanes
    for (int wb = (blockIdx.x * wpb + warp) * SPW; wb < nwork; wb += gridDim.x * wpb * SPW) {
        int w = wb + q;
        bool has = w < nwork;
        int ic = has ? worklist[w] : 0;
        int i = has ? cpts[ic] : 0;
        int np = has ? npat[ic] : 0;
        double *M = gbuf ? gbuf + (has ? goff[w] : 0)
                         : smem + ((size_t)warp * SPW + q) * ((size_t)nmax * nmax + 4 * nmax);
        double *y = M + (size_t)np * np;
        double *rv = y + np;                  // pivot reciprocals
        int *pat = (int *)(rv + np);
        int *piv = pat + np;
        int *rl = piv + np;                   // rows below the pivot with a nonzero multiplier
        if (has) {
            const int *cp = cand + candptr[ic];
            for (int t = g; t < np; t += G) { pat[t] = cp[t]; y[t] = -0.0; }
            for (int idx = g; idx < np * np; idx += G) M[idx] = 0.0;
        }
        __syncwarp();
        if (has) {
            // M[r][c] = a(pat[c], pat[r]): lane per pattern row, one pass over it, the
            // loads of four entries issued before their lookups
            for (int c = g; c < np; c += G) {
                const int j = pat[c], p1 = rowptr[j + 1];
                for (int p = rowptr[j]; p < p1; p += 4) {
                    int cc[4];
                    double vv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        cc[u] = p + u < p1 ? col[p + u] : -1;
                        vv[u] = p + u < p1 ? val[p + u] : 0.0;
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        if (cc[u] < 0) continue;
                        const int r = pat_find(pat, np, cc[u]);
                        if (r >= 0) M[r * np + c] = vv[u];
                    }
                }
            }
            for (int p = rowptr[i] + g; p < rowptr[i + 1]; p += G) {
                int r = pat_find(pat, np, col[p]);
                if (r >= 0) y[r] = -val[p];
            }
        }
        __syncwarp();
        long long mxb = 0;
        for (int idx = g; idx < np * np; idx += G) mxb = max(mxb, absbits(M[idx]));
        for (int o = G / 2; o > 0; o >>= 1) mxb = max(mxb, __shfl_xor_sync(FULL, mxb, o, G));
        long long tinyb = absbits(1e-14 * __longlong_as_double(mxb));
        int kmax = np;
        for (int o = 16; o > 0; o >>= 1) kmax = max(kmax, __shfl_xor_sync(FULL, kmax, o));
        bool singular = false;
        for (int k = 0; k < kmax; ++k) {
            bool act = k < np && !singular;
            long long bv = -1;
            int br = k;
            bool nzb = false;   // a nonzero below the diagonal among this lane's rows
            if (act)
                for (int r = k + g; r < np; r += G) {
                    long long v = absbits(M[r * np + k]);
                    if (r > k && v != 0) nzb = true;
                    if (v > bv) { bv = v; br = r; }
                }
            // Most columns have nothing below the diagonal: when no group of the warp has,
            // every pivot stays on the diagonal (the only candidate that is not zero,
            // held by the group's first lane) and the step has no multipliers to compute
            // and nothing to update.
            const bool any_nz = __ballot_sync(FULL, nzb) != 0u;
            if (any_nz) {
                for (int o = G / 2; o > 0; o >>= 1) {
                    long long ov = __shfl_xor_sync(FULL, bv, o, G);
                    int orr = __shfl_xor_sync(FULL, br, o, G);
                    if (ov > bv || (ov == bv && orr < br)) { bv = ov; br = orr; }
                }
            } else {
                bv = __shfl_sync(FULL, bv, q * G);
                br = k;
            }
            if (act && !(bv > tinyb)) { singular = true; act = false; }
            if (act) {
                if (g == 0) piv[k] = br;
                if (br != k)
                    for (int c = g; c < np; c += G) {
                        double t = M[k * np + c];
                        M[k * np + c] = M[br * np + c];
                        M[br * np + c] = t;
                    }
            }
            __syncwarp();
            // multipliers, and the list of rows whose multiplier is not zero: a zero
            // multiplier's update adds exact zeros, so those rows are skipped, as in the
            // reference LU (in the local systems of these operators most multipliers are
            // zero).  The bound on the rows below the pivot is uniform over the warp, so
            // every lane reaches each ballot.
            // (a zero entry's multiplier is the signed zero a * rd gives, set with
            // integer operations; the others are computed for the listed rows only)
            int m = 0;
            if (!any_nz) {
                // only zeros below: their multipliers are those zeros, with the sign
                // flipped under a negative pivot (the sign of 1 / pivot, so no division
                // here: the reciprocals of such pivots are taken together after the
                // elimination)
                const double pk = act ? M[k * np + k] : 0.0;   // k < np only for an active group
                if (act && __double_as_longlong(pk) < 0)
                    for (int r = k + 1 + g; r < np; r += G) M[r * np + k] = zero_times(M[r * np + k], pk);
                __syncwarp();
                continue;
            }
            // the pivot's reciprocal: one lane of the group divides, the others take it
            double rd = 0.0;
            if (act && g == 0) rd = pivot_recip(M[k * np + k]);
            rd = __shfl_sync(FULL, rd, q * G);
            for (int j0 = 0; j0 < kmax - k - 1; j0 += G) {
                const int r = k + 1 + j0 + g;
                bool nzr = false;
                if (act && r < np) {
                    const double a = M[r * np + k];
                    nzr = !is_zero_bits(a);
                    if (!nzr) M[r * np + k] = zero_times(a, rd);
                }
                const unsigned msk = __ballot_sync(FULL, nzr) & gmask;
                if (nzr) rl[m + __popc(msk & ((1u << lane) - 1u))] = r;
                m += __popc(msk);
            }
            __syncwarp();
            if (act)
                for (int t = g; t < m; t += G) {
                    const double l = M[rl[t] * np + k] * rd;
                    M[rl[t] * np + k] = l;
                    if (is_zero_bits(l)) rl[t] = -1;   // underflowed to zero: skipped too
                }
            __syncwarp();
            if (act) {
                // lane g updates entries g, g + G, ... of the m x wd block (listed rows,
                // trailing columns) in row-major order (the fewest FP64 instructions:
                // every lane busy until the last entries), four entries per pass with all
                // their loads issued before the updates; (list index, column) advance by
                // (G / wd, G % wd) per entry with at most one carry, so no division per
                // entry
                const int wd = np - k - 1;
                if (wd > 0 && m > 0) {
                    const int tot = m * wd;
                    const int dr = G / wd, dc = G - dr * wd;
                    int r = g / wd, c = g - r * wd;
                    for (int e = g; e < tot; e += 4 * G) {
                        int Ro[4], Co[4];
                        bool ok[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int rr = e + u * G < tot ? rl[r] : -1;
                            ok[u] = rr >= 0;
                            Ro[u] = ok[u] ? rr * np : 0;
                            Co[u] = k + 1 + c;
                            r += dr;
                            c += dc;
                            if (c >= wd) { c -= wd; ++r; }
                        }
                        double a[4], b[4], mv[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            if (ok[u]) { a[u] = M[Ro[u] + k]; b[u] = M[k * np + Co[u]]; mv[u] = M[Ro[u] + Co[u]]; }
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            if (ok[u]) M[Ro[u] + Co[u]] = fma(-a[u], b[u], mv[u]);
                    }
                }
            }
            __syncwarp();
        }
        bool solve = has && !singular && np > 0;
        // every pivot's reciprocal for the back substitution, G at a time (the same
        // values the elimination took for its multipliers)
        if (solve)
            for (int k = g; k < np; k += G) rv[k] = pivot_recip(M[k * np + k]);
        if (solve && g == 0)
            for (int k = 0; k < np; ++k)
                if (piv[k] != k) { double t = y[k]; y[k] = y[piv[k]]; y[piv[k]] = t; }
        __syncwarp();
        for (int k = 0; k < kmax; ++k) {
            if (solve && k < np) {
                double yk = y[k];
                for (int r = k + 1 + g; r < np; r += G) y[r] = fma(-M[r * np + k], yk, y[r]);
            }
            __syncwarp();
        }
        for (int k = kmax - 1; k >= 0; --k) {
            if (solve && k < np && g == 0) y[k] = times_recip(y[k], rv[k]);
            __syncwarp();
            if (solve && k < np) {
                double yk = y[k];
                for (int r = g; r < k; r += G) y[r] = fma(-M[r * np + k], yk, y[r]);
            }
            __syncwarp();
        }
        long long zmb = 0;
        if (solve)
            for (int t = g; t < np; t += G) zmb = max(zmb, absbits(y[t]));
        for (int o = G / 2; o > 0; o >>= 1) zmb = max(zmb, __shfl_xor_sync(FULL, zmb, o, G));
        double thr = phi_R * __longlong_as_double(zmb);
        int kept = 0;
        int base = has ? zrowptr[ic] : 0;
        int tmax = np;
        for (int o = 16; o > 0; o >>= 1) tmax = max(tmax, __shfl_xor_sync(FULL, tmax, o));
        // keep in ascending order: ballot-compacted write within the group
        for (int t0 = 0; t0 < tmax; t0 += G) {
            int t = t0 + g;
            bool k_ = solve && t < np && !(phi_R > 0.0 && fabs(y[t]) < thr);
            unsigned msk = __ballot_sync(FULL, k_) & gmask;
            if (k_) {
                int off = kept + __popc(msk & ((1u << lane) - 1u));
                zcol[base + off] = pat[t];
                zval[base + off] = y[t];
            }
            kept += __popc(msk);
        }
        if (has && g == 0) {
            if (singular) atomicAdd(&nsing_dir[rowdir[i]], 1);
            keep[ic] = solve ? kept : 0;
        }
        __syncwarp();
    }
}

__global__ void k_compact_rows(int nrows, const int *oldptr, const int *newptr, const int *col_in,
                               const double *val_in, int *col_out, double *val_out) {
    long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int r = (int)(tid >> 3), g = (int)(tid & 7);
    if (r >= nrows) return;
    int o = oldptr[r], nn = newptr[r], cnt = newptr[r + 1] - newptr[r];
    for (int t = g; t < cnt; t += 8) { col_out[nn + t] = col_in[o + t]; val_out[nn + t] = val_in[o + t]; }
}

// ---- RAP ---------------------------------------------------------------------
// Thread per fine row k: (AP)[k,c] accumulated in ascending l order, then
// sorted by c.  Rows of up to 64 entries work in local arrays, longer rows in
// their output slots.
__global__ void k_ap(int n, const int *rowptr, const int *col, const double *val, const int *pmap,
                     const int8_t *cf, int *aplen, int *apcol, double *apval) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    if (cf[k] == CF_COARSEST) { aplen[k] = 0; return; }
    int s = rowptr[k], e = rowptr[k + 1];
    int len = 0;
    if (e - s <= 64) {
        int lc[64];
        double lv[64];
        for (int p = s; p < e; ++p) {
            int c = pmap[col[p]];
            if (c < 0) continue;
            int t = 0;
            while (t < len && lc[t] != c) ++t;
            if (t == len) { lc[t] = c; lv[t] = 0.0; ++len; }
            lv[t] = lv[t] + val[p];
        }
        for (int a = 1; a < len; ++a) {
            int c = lc[a];
            double v = lv[a];
            int b = a;
            while (b > 0 && lc[b - 1] > c) { lc[b] = lc[b - 1]; lv[b] = lv[b - 1]; --b; }
            lc[b] = c;
            lv[b] = v;
        }
        for (int t = 0; t < len; ++t) { apcol[s + t] = lc[t]; apval[s + t] = lv[t]; }
        aplen[k] = len;
        return;
    }
    for (int p = s; p < e; ++p) {
        int c = pmap[col[p]];
        if (c < 0) continue;
        int t = 0;
        while (t < len && apcol[s + t] != c) ++t;
        if (t == len) { apcol[s + t] = c; apval[s + t] = 0.0; ++len; }
        apval[s + t] = apval[s + t] + val[p];
    }
    for (int a = 1; a < len; ++a) {
        int c = apcol[s + a];
        double v = apval[s + a];
        int b = a;
        while (b > 0 && apcol[s + b - 1] > c) { apcol[s + b] = apcol[s + b - 1]; apval[s + b] = apval[s + b - 1]; --b; }
        apcol[s + b] = c;
        apval[s + b] = v;
    }
    aplen[k] = len;
}

__global__ void k_rap_bound(int nc, const int *cpts, const int *zrowptr, const int *zcol, const int *aplen, int *U) {
    int ic = blockIdx.x * blockDim.x + threadIdx.x;
    if (ic >= nc) return;
    int u = aplen[cpts[ic]];
    for (int t = zrowptr[ic]; t < zrowptr[ic + 1]; ++t) u += aplen[zcol[t]];
    U[ic] = u;
}

__device__ __forceinline__ unsigned hslot(int c, unsigned mask) { return ((unsigned)c * 2654435761u) & mask; }

// G lanes per coarse row (32/G rows per warp).  Table: keys (int, -1 empty)
// and values, in shared memory (hcap slots per row, sized to the row's bin) or
// in global scratch (cap per row given by gptr).  Output: sorted, filtered
// entries at ucol/uval[uptr[ic]...], count in cnt[ic].  Magnitude maxima use
// integer keys; the phi_A filter costs nothing when it is off (filt == 0).
// A row's table has the first power of two >= its bound U (at least 64) slots:
// U bounds the row's distinct columns, so linear probing always finds a slot, and
// on the transport operators the distinct columns are on average 20-55% of U, so
// tables stay about half full or less.  Each slot's additions follow the R-row
// order whatever the table size, so the size changes no bit of the result.
template <int G, bool GLOBAL_TABLE>
__global__ void k_rap(int nrows_work, const int *worklist, const int *cpts, const int *zrowptr, const int *zcol,
                      const double *zval, const int *aprow, const int *aplen, const int *apcol, const double *apval,
                      const int *uptr, const int *U, int filt, double phiA, int *cnt, int *ucol, double *uval, int hcap,
                      const long long *gptr, int *gkeys, double *gvals, int *overflow, int *err) {
    extern __shared__ double smem2[];
    const unsigned FULL = 0xffffffffu;
    constexpr int SPW = 32 / G;
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int g = lane % G, q = lane / G;
    int wpb = blockDim.x >> 5;
    unsigned gmask = (G == 32) ? FULL : (((1u << (G & 31)) - 1u) << (q * G));
    for (int wb = (blockIdx.x * wpb + warp) * SPW; wb < nrows_work; wb += gridDim.x * wpb * SPW) {
        int w = wb + q;
        bool has = w < nrows_work;
        int ic = has ? worklist[w] : 0;
        int *keys = nullptr;
        double *vals = nullptr;
        int cap = 0;
        if (has) {
            if (GLOBAL_TABLE) {
                long long off = gptr[w];
                cap = (int)(gptr[w + 1] - off);
                keys = gkeys + off;
                vals = gvals + off;
            } else {
                int slot = warp * SPW + q;
                vals = smem2 + (size_t)slot * hcap;
                keys = (int *)(smem2 + (size_t)wpb * SPW * hcap) + (size_t)slot * hcap;
                if (U[ic] > hcap) {
                    if (g == 0) { cnt[ic] = -1; atomicAdd(overflow, 1); }
                    has = false;
                } else {
                    cap = 64;
                    while (cap < U[ic]) cap <<= 1;
                }
            }
        }
        unsigned mask = (unsigned)cap - 1u;
        for (int t = g; t < cap; t += G) keys[t] = -1;
        __syncwarp();
        int i = has ? cpts[ic] : 0;
        int z0 = has ? zrowptr[ic] : 0, z1 = has ? zrowptr[ic + 1] : 0;
        int nr = has ? z1 - z0 + 1 : 0;   // R row entries, identity included
        int nrmax = nr;
        for (int o = 16; o > 0; o >>= 1) nrmax = max(nrmax, __shfl_xor_sync(FULL, nrmax, o));
        // The R row in ascending column order (the identity at column i); each step's
        // chain of loads (its column, then its AP row, then the AP row's first entry
        // of this lane) is issued one step ahead, while the previous step's entries
        // go into the table.  The additions into each slot keep the R-row order.
        bool placed = false;
        int t = z0;
        int zc = (t < z1) ? zcol[t] : 0x7fffffff;   // the next Z column
        auto advance = [&](int &k, double &r) {
            if (!placed && zc > i) { k = i; r = 1.0; placed = true; }
            else { k = zc; r = zval[t]; ++t; zc = (t < z1) ? zcol[t] : 0x7fffffff; }
        };
        int k_c = 0, a_c = 0, l_c = 0, c_c = 0;
        double r_c = 0.0, v_c = 0.0;
        if (nr > 0) {
            advance(k_c, r_c);
            a_c = aprow[k_c];
            l_c = aplen[k_c];
            if (g < l_c) { c_c = apcol[a_c + g]; v_c = apval[a_c + g]; }
        }
        for (int step = 0; step < nrmax; ++step) {
            int k_n = 0, a_n = 0, l_n = 0, c_n = 0;
            double r_n = 0.0, v_n = 0.0;
            if (step + 1 < nr) {
                advance(k_n, r_n);
                a_n = aprow[k_n];
                l_n = aplen[k_n];
                if (g < l_n) { c_n = apcol[a_n + g]; v_n = apval[a_n + g]; }
            }
            if (step < nr) {
                const double r = r_c;
                const int a0 = a_c, al = l_c;
                for (int qq = g; qq < al; qq += G) {
                    int c;
                    double v;
                    if (qq == g) { c = c_c; v = v_c; }
                    else { c = apcol[a0 + qq]; v = apval[a0 + qq]; }
                    unsigned hs = hslot(c, mask);
                    int probes = 0;
                    bool ok = false;
                    while (probes++ < cap) {
                        int prev = atomicCAS(&keys[hs], -1, c);
                        if (prev == -1) { vals[hs] = 0.0; ok = true; break; }
                        if (prev == c) { ok = true; break; }
                        hs = (hs + 1) & mask;
                    }
                    if (ok) vals[hs] = fma(r, v, vals[hs]);
                    else atomicOr(err, DERR_HASH_OVERFLOW);
                }
            }
            __syncwarp();
            k_c = k_n; r_c = r_n; a_c = a_n; l_c = l_n; c_c = c_n; v_c = v_n;
        }
        // compact to the scratch output (unsorted), then rank-sort back into the table
        int base = has ? uptr[ic] : 0;
        int m = 0;
        int capmax = cap;
        for (int o = 16; o > 0; o >>= 1) capmax = max(capmax, __shfl_xor_sync(FULL, capmax, o));
        for (int s0 = 0; s0 < capmax; s0 += G) {
            int sl = s0 + g;
            bool occ = sl < cap && keys[sl] >= 0;
            unsigned msk = __ballot_sync(FULL, occ) & gmask;
            if (occ) {
                int off = m + __popc(msk & ((1u << lane) - 1u));
                ucol[base + off] = keys[sl];
                uval[base + off] = vals[sl];
            }
            m += __popc(msk);
        }
        __syncwarp();
        for (int e = g; e < m; e += G) {
            int ce = ucol[base + e];
            int rank = 0;
            for (int f = 0; f < m; ++f) rank += ucol[base + f] < ce;
            keys[rank] = ce;
            vals[rank] = uval[base + e];
        }
        __syncwarp();
        int mmax = m;
        for (int o = 16; o > 0; o >>= 1) mmax = max(mmax, __shfl_xor_sync(FULL, mmax, o));
        double thr = 0.0;
        if (filt) {
            long long mxb = 0;
            for (int e = g; e < m; e += G)
                if (keys[e] != ic) mxb = max(mxb, absbits(vals[e]));
            for (int o = G / 2; o > 0; o >>= 1) mxb = max(mxb, __shfl_xor_sync(FULL, mxb, o, G));
            thr = phiA * __longlong_as_double(mxb);
        }
        int kept = 0;
        for (int e0 = 0; e0 < mmax; e0 += G) {
            int e = e0 + g;
            bool k_ = e < m && !(filt && keys[e] != ic && fabs(vals[e]) < thr);
            unsigned msk = __ballot_sync(FULL, k_) & gmask;
            if (k_) {
                int off = kept + __popc(msk & ((1u << lane) - 1u));
                ucol[base + off] = keys[e];
                uval[base + off] = vals[e];
            }
            kept += __popc(msk);
        }
        if (has && g == 0) cnt[ic] = kept;
        __syncwarp();
    }
}

__global__ void k_gather_int(int n, const int *src, const int *idx, int *out) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) out[k] = src[idx[k]];
}

__global__ void k_gather_rowdir(int nc, const int *cpts, const int *rowdir, int *rowdir_c) {
    int ic = blockIdx.x * blockDim.x + threadIdx.x;
    if (ic < nc) rowdir_c[ic] = rowdir[cpts[ic]];
}

__global__ void k_rowlen_dir(int n, const int *rowptr, const int *rowdir, unsigned long long *nnzdir) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool valid = i < n;
    int d = valid ? rowdir[i] : 0;
    add_by_dir<unsigned long long>(nnzdir, d, valid ? (unsigned long long)(rowptr[i + 1] - rowptr[i]) : 0ULL, valid);
}

__global__ void k_fill_int8(int n, int8_t *a, int8_t v) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

__global__ void k_fill_int(int n, int *a, int v) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

__device__ __forceinline__ int rap_bin(int u) { return u <= 128 ? 0 : u <= 512 ? 1 : u <= 2048 ? 2 : 3; }



__global__ void k_overflow_caps(int nover, const int *list, const int *U, long long *capw) {
    int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nover) return;
    long long c = 64;
    while (c < (long long)U[list[w]]) c <<= 1;
    capw[w] = c;
}

__global__ void k_big_rows(int nbig, const int *list, const int *npat, long long *goff) {
    int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nbig) return;
    long long np = npat[list[w]];
    goff[w] = np * np + 4 * np;
}


__global__ void k_lair_classes(int nc, const int *npat, int8_t *cls) {
    int ic = blockIdx.x * blockDim.x + threadIdx.x;
    if (ic < nc) cls[ic] = (int8_t)lair_class(npat[ic]);
}

__global__ void k_rap_classes(int nc, const int *U, int8_t *cls) {
    int ic = blockIdx.x * blockDim.x + threadIdx.x;
    if (ic < nc) cls[ic] = (int8_t)rap_bin(U[ic]);
}

template <class T>
void d2h(T *h, const T *d, size_t count, cudaStream_t s) {
    PR_CUDA(cudaMemcpyAsync(h, d, count * sizeof(T), cudaMemcpyDeviceToHost, s));
    PR_CUDA(cudaStreamSynchronize(s));
}

// Rows 0..n-1 grouped by class (ascending row order inside each class):
// list[start[c] .. start[c] + count[c]).  A counting sort, deterministic: per
// block of PART_BS rows the rows of each class (counted by warp ballots), an
// exclusive scan over (class, block), and a scatter at each row's rank among the
// rows of its class before it.  One host read (the class counts).
constexpr int PART_BS = 256;
constexpr int PART_MAXC = 16;

__global__ void __launch_bounds__(PART_BS) k_class_hist(int n, const int8_t *cls, int nclass, int nblk, int *hist) {
    __shared__ int wc[PART_BS / 32][PART_MAXC];
    const int i = blockIdx.x * PART_BS + threadIdx.x;
    const int c = (i < n && cls[i] >= 0 && cls[i] < nclass) ? cls[i] : -1;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = 0; k < nclass; ++k) {
        const unsigned m = __ballot_sync(0xffffffffu, c == k);
        if (lane == 0) wc[w][k] = __popc(m);
    }
    __syncthreads();
    if ((int)threadIdx.x < nclass) {
        int t = 0;
        for (int ww = 0; ww < PART_BS / 32; ++ww) t += wc[ww][threadIdx.x];
        hist[threadIdx.x * nblk + blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(PART_BS) k_class_scatter(int n, const int8_t *cls, int nclass, int nblk,
                                                           const int *off, int *list) {
    __shared__ int wc[PART_BS / 32][PART_MAXC];
    const int i = blockIdx.x * PART_BS + threadIdx.x;
    const int c = (i < n && cls[i] >= 0 && cls[i] < nclass) ? cls[i] : -1;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int rank_in_warp = 0;
    for (int k = 0; k < nclass; ++k) {
        const unsigned m = __ballot_sync(0xffffffffu, c == k);
        if (lane == 0) wc[w][k] = __popc(m);
        if (c == k) rank_in_warp = __popc(m & ((1u << lane) - 1u));
    }
    __syncthreads();
    if (c < 0) return;
    int before = 0;
    for (int ww = 0; ww < w; ++ww) before += wc[ww][c];
    list[off[c * nblk + blockIdx.x] + before + rank_in_warp] = i;
}

__global__ void k_class_counts(int nclass, int nblk, const int *off, int *out) {
    const int c = threadIdx.x;
    if (c <= nclass) out[c] = off[c * nblk];   // class starts, and the total
}

void partition_by_class(const int8_t *cls, int n, int nclass, int *list, int *start, int *count, cudaStream_t s) {
    PR_REQUIRE(nclass >= 1 && nclass <= PART_MAXC, PAIR_ERR_DEVICE, "partition_by_class: too many classes");
    if (n <= 0) {
        for (int c = 0; c < nclass; ++c) { start[c] = 0; count[c] = 0; }
        return;
    }
    const int nblk = (int)blocks_for(n, PART_BS);
    const int nh = nclass * nblk;
    int *hist = dmalloc<int>(nh, s), *off = dmalloc<int>(nh + 1, s), *cs = dmalloc<int>(nclass + 1, s);
    k_class_hist<<<nblk, PART_BS, 0, s>>>(n, cls, nclass, nblk, hist);
    PR_LAUNCH();
    scan_exclusive(hist, off, nh, s, false);
    k_class_scatter<<<nblk, PART_BS, 0, s>>>(n, cls, nclass, nblk, off, list);
    PR_LAUNCH();
    k_class_counts<<<1, 32, 0, s>>>(nclass, nblk, off, cs);
    PR_LAUNCH();
    int h[PART_MAXC + 1];
    d2h(h, cs, nclass + 1, s);
    for (int c = 0; c < nclass; ++c) { start[c] = h[c]; count[c] = h[c + 1] - h[c]; }
    dfree(hist, s);
    dfree(off, s);
    dfree(cs, s);
}

__global__ void k_split_len(int n, const int *srow, const int *rowptr, int *len) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) {
        int i = srow[k];
        len[k] = rowptr[i + 1] - rowptr[i];
    }
}

// entries of split row k (row srow[k]) copied to sptr[k].., eight lanes per row
template <class T>
__global__ void k_split_copy(int n, const int *srow, const int *rowptr, const int *col, const double *val,
                             const int *sptr, int *scol, T *sval) {
    long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int k = (int)(tid >> 3), g = (int)(tid & 7);
    if (k >= n) return;
    int i = srow[k];
    int a = rowptr[i], len = rowptr[i + 1] - a, d = sptr[k];
    for (int q = g; q < len; q += 8) {
        scol[d + q] = col[a + q];
        sval[d + q] = (T)val[a + q];
    }
}

// ---- sliced ELL (SELL-32) copies for the V-cycle's row dot products -------------
// Rows are taken in windows of 256 and ordered inside each window by decreasing
// length (ties by position); every 32 consecutive positions form a slice whose
// entries are stored column-major with the slice's first (longest) row setting its
// width: entry j of the row at lane t of slice s sits at ptr[s] + 32 j + t.
constexpr int SELL_WIN = 256;

// rows[q] (or q when rows is null), q < nr: CSR row of list position q
__global__ void k_sell_rank(int nr, const int *rows, const int *rowptr, int *out_row, int *out_len) {
    __shared__ int sl[SELL_WIN];
    const int t = threadIdx.x, q = blockIdx.x * SELL_WIN + t;
    const int r = q < nr ? (rows ? rows[q] : q) : -1;
    const int len = r >= 0 ? rowptr[r + 1] - rowptr[r] : -1;
    sl[t] = len;
    __syncthreads();
    int rank = 0;
    for (int u = 0; u < SELL_WIN; ++u) {
        const int lu = sl[u];
        rank += (lu > len || (lu == len && u < t)) ? 1 : 0;
    }
    const int pos = blockIdx.x * SELL_WIN + rank;
    out_row[pos] = r;
    out_len[pos] = len > 0 ? len : 0;
}

__global__ void k_sell_width(int ns, const int *len, int *w32) {
    int sl = blockIdx.x * blockDim.x + threadIdx.x;
    if (sl < ns) w32[sl] = 32 * len[32 * sl];
}

template <class T>
__global__ void k_sell_fill(int npos, const int *prow, const int *plen, const int *sptr, const int *rowptr,
                            const int *col, const double *val, int *scol, T *sval) {
    int pos = blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= npos) return;
    const int r = prow[pos];
    if (r < 0) return;
    const int a = rowptr[r], len = plen[pos];
    const int base = sptr[pos >> 5] + (pos & 31);
    for (int j = 0; j < len; ++j) {
        scol[base + 32 * j] = col[a + j];
        sval[base + 32 * j] = (T)val[a + j];
    }
}

// 16-bit column offsets: an entry's column minus its row, when every stored entry
// of a store fits (the relaxation stores of the coarse levels: their stencils stay
// within a few mesh planes of the row); the padding slots are never read
// offsets are taken from the row's own index, or (rowbase, the restriction's Z
// rows) from the fine row of its coarse point
__global__ void k_sell_off_check(int npos, const int *prow, const int *plen, const int *sptr, const int *scol,
                                 const int *rowbase, int *bad) {
    const int pos = blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= npos) return;
    const int q = prow[pos];
    if (q < 0) return;
    const int r = rowbase ? rowbase[q] : q;
    const int len = plen[pos], base = sptr[pos >> 5] + (pos & 31);
    for (int j = 0; j < len; ++j) {
        const int off = scol[base + 32 * j] - r;
        if (off < -32768 || off > 32767) { atomicOr(bad, 1); return; }
    }
}

__global__ void k_sell_to16(int npos, const int *prow, const int *plen, const int *sptr, const int *scol,
                            const int *rowbase, short *col16) {
    const int pos = blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= npos) return;
    const int q = prow[pos];
    if (q < 0) return;
    const int r = rowbase ? rowbase[q] : q;
    const int len = plen[pos], base = sptr[pos >> 5] + (pos & 31);
    for (int j = 0; j < len; ++j) col16[base + 32 * j] = (short)(scol[base + 32 * j] - r);
}

void sell_compress_cols(Hier &h, Sell &S, const int *rowbase = nullptr) {
    if (S.nrows <= 0 || !S.col) return;
    cudaStream_t s = h.stream;
    const int BS = 256;
    int *bad = dmalloc<int>(1, s);
    PR_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    k_sell_off_check<<<blocks_for(S.npos, BS), BS, 0, s>>>(S.npos, S.row, S.len, S.ptr, S.col, rowbase, bad);
    PR_LAUNCH();
    int hb = 0;
    d2h(&hb, bad, 1, s);
    dfree(bad, s);
    if (hb) return;
    S.col16 = dmalloc<short>(std::max<long long>(S.nnz, 1), s);
    k_sell_to16<<<blocks_for(S.npos, BS), BS, 0, s>>>(S.npos, S.row, S.len, S.ptr, S.col, rowbase, S.col16);
    PR_LAUNCH();
    dfree(S.col, s);
    S.col = nullptr;
}

// SELL copy of nr rows of a CSR matrix (list rows, or rows 0..nr-1), values in the
// V-cycle's precision
void build_sell(Hier &h, Sell &S, const int *rows, int nr, const int *rowptr, const int *col, const double *val) {
    cudaStream_t s = h.stream;
    const int BS = 256;
    S.nrows = nr;
    if (nr <= 0) return;
    const int nwin = (nr + SELL_WIN - 1) / SELL_WIN;
    S.npos = nwin * SELL_WIN;
    const int ns = S.npos / 32;
    S.row = dmalloc<int>(S.npos, s);
    S.len = dmalloc<int>(S.npos, s);
    k_sell_rank<<<nwin, SELL_WIN, 0, s>>>(nr, rows, rowptr, S.row, S.len);
    PR_LAUNCH();
    int *w32 = dmalloc<int>(ns, s);
    k_sell_width<<<blocks_for(ns, BS), BS, 0, s>>>(ns, S.len, w32);
    PR_LAUNCH();
    S.ptr = dmalloc<int>(ns + 1, s);
    S.nnz = scan_exclusive(w32, S.ptr, ns, s);
    dfree(w32, s);
    S.col = dmalloc<int>(std::max<long long>(S.nnz, 1), s);
    if (h.prm.precision >= 1) {
        S.val = dmalloc<float>(std::max<long long>(S.nnz, 1), s);
        k_sell_fill<float><<<blocks_for(S.npos, BS), BS, 0, s>>>(S.npos, S.row, S.len, S.ptr, rowptr, col, val,
                                                                 S.col, (float *)S.val);
    } else {
        S.val = dmalloc<double>(std::max<long long>(S.nnz, 1), s);
        k_sell_fill<double><<<blocks_for(S.npos, BS), BS, 0, s>>>(S.npos, S.row, S.len, S.ptr, rowptr, col, val,
                                                                  S.col, (double *)S.val);
    }
    PR_LAUNCH();
}

// CF split of one level (see Level): the row order [F | C | coarsest], SELL copies
// of the F and C rows (with_fc) and a CSR copy of the coarsest rows with the
// coarsest segments' positions in it
void build_split(Hier &h, Level &L, bool with_fc) {
    cudaStream_t s = h.stream;
    const int BS = 256;
    const int n = L.n;
    const size_t es = h.prm.precision >= 1 ? sizeof(float) : sizeof(double);
    int st[3] = {0, 0, 0}, cnt[3] = {0, 0, 0};
    L.srow = dmalloc<int>(std::max(n, 1), s);
    partition_by_class(L.cf, n, 3, L.srow, st, cnt, s);
    PR_REQUIRE(cnt[0] + cnt[1] + cnt[2] == n, PAIR_ERR_DEVICE, "CF split does not cover the level's rows");
    L.nF = cnt[0];
    L.nC = cnt[1];
    const int kX = L.nF + L.nC, nx = n - kX;
    if (with_fc) {
        build_sell(h, L.sF, L.srow, L.nF, L.rowptr, L.col, L.val);
        build_sell(h, L.sC, L.srow + L.nF, L.nC, L.rowptr, L.col, L.val);
        sell_compress_cols(h, L.sF);
        sell_compress_cols(h, L.sC);
    }
    if (nx > 0) {
        int *len = dmalloc<int>(nx, s);
        k_split_len<<<blocks_for(nx, BS), BS, 0, s>>>(nx, L.srow + kX, L.rowptr, len);
        PR_LAUNCH();
        L.sptr = dmalloc<int>(nx + 1, s);
        long long tot = scan_exclusive(len, L.sptr, nx, s);
        dfree(len, s);
        L.scol = dmalloc<int>(std::max<long long>(tot, 1), s);
        L.sval = dmalloc<char>(std::max<long long>(tot, 1) * es, s);
        if (h.prm.precision >= 1)
            k_split_copy<float><<<blocks_for((long long)nx * 8, BS), BS, 0, s>>>(
                nx, L.srow + kX, L.rowptr, L.col, L.val, L.sptr, L.scol, (float *)L.sval);
        else
            k_split_copy<double><<<blocks_for((long long)nx * 8, BS), BS, 0, s>>>(
                nx, L.srow + kX, L.rowptr, L.col, L.val, L.sptr, L.scol, (double *)L.sval);
        PR_LAUNCH();
    }
    // coarsest segments are whole matrices, ascending in row order, so each one is a
    // contiguous run of the coarsest group; positions relative to the group's start
    std::vector<int> s0;
    long long pos = 0, prev = -1;
    for (int d = 0; d < h.ndir; ++d)
        if (L.nrows[d] > 0 && L.coarsest[d]) {
            PR_REQUIRE(L.row0[d] > prev, PAIR_ERR_DEVICE, "coarsest segments out of row order");
            prev = L.row0[d];
            s0.push_back((int)pos);
            pos += L.nrows[d];
        }
    PR_REQUIRE(pos == nx, PAIR_ERR_DEVICE, "coarsest rows differ from the coarsest segments");
    PR_REQUIRE((int)s0.size() == L.n_cseg, PAIR_ERR_DEVICE, "coarsest segment count mismatch");
    // a segment too large for the one-CTA shared-memory sweeps: SELL copy of every
    // coarsest row of the level, swept grid-wide
    bool big = false;
    for (int d = 0; d < h.ndir; ++d)
        if (L.nrows[d] > 0 && L.coarsest[d]) {
            const size_t nr = (size_t)L.nrows[d], nz = (size_t)L.nnzdir[d];
            big |= nz * (es + sizeof(int)) + 4 * nr * es + (nr + 1) * sizeof(int) > (size_t)CS_SMEM;
        }
    if (big) {
        build_sell(h, L.sX, L.srow + kX, nx, L.rowptr, L.col, L.val);
        sell_compress_cols(h, L.sX);
    }
    if (!s0.empty()) {
        L.d_cseg_s0 = dmalloc<int>(s0.size(), s);
        PR_CUDA(cudaMemcpyAsync(L.d_cseg_s0, s0.data(), sizeof(int) * s0.size(), cudaMemcpyHostToDevice, s));
        PR_CUDA(cudaStreamSynchronize(s));
    }
}

}  // namespace

void free_level(Level &L, cudaStream_t s) {
    void *ptrs[] = {L.rowptr, L.col, L.val, L.dinv, L.dinv32, L.cf, L.pmap, L.rowdir, L.cpts,
                    L.zrowptr, L.zcol, L.zval, L.d_row0, L.d_cseg_row0, L.d_cseg_n,
                    L.srow, L.sptr, L.scol, L.sval, L.d_cseg_s0,
                    L.sF.ptr, L.sF.row, L.sF.len, L.sF.col, L.sF.col16, L.sF.val, L.sC.ptr, L.sC.row, L.sC.len,
                    L.sC.col, L.sC.col16, L.sC.val, L.sZ.ptr, L.sZ.row, L.sZ.len, L.sZ.col, L.sZ.col16, L.sZ.val,
                    L.sX.ptr, L.sX.row, L.sX.len, L.sX.col, L.sX.col16, L.sX.val, L.vb, L.vx, L.vxn, L.vy};
    for (void *p : ptrs) dfree(p, s);
    L = Level();
}

static void finish_segments(Hier &h, Level &L) {
    cudaStream_t s = h.stream;
    std::vector<int> r0, nn;
    for (int d = 0; d < h.ndir; ++d)
        if (L.nrows[d] > 0 && L.coarsest[d]) { r0.push_back(L.row0[d]); nn.push_back(L.nrows[d]); }
    L.n_cseg = (int)r0.size();
    if (L.n_cseg) {
        L.d_cseg_row0 = dmalloc<int>(L.n_cseg, s);
        L.d_cseg_n = dmalloc<int>(L.n_cseg, s);
        PR_CUDA(cudaMemcpyAsync(L.d_cseg_row0, r0.data(), sizeof(int) * r0.size(), cudaMemcpyHostToDevice, s));
        PR_CUDA(cudaMemcpyAsync(L.d_cseg_n, nn.data(), sizeof(int) * nn.size(), cudaMemcpyHostToDevice, s));
        PR_CUDA(cudaStreamSynchronize(s));
    }
}

void build_hierarchy(Hier &h) {
    cudaStream_t s = h.stream;
    const air_params &prm = h.prm;
    const int ND = h.ndir;
    const int BS = 256;
    int *d_count = dmalloc<int>(1, s);
    char *dwork = dmalloc<char>(ND, s);
    char *dcont = dmalloc<char>(ND, s);
    int *dnc = dmalloc<int>(ND, s);
    long long *dnnz = dmalloc<long long>(ND, s);
    cudaEvent_t ev[4];
    for (auto &e : ev) PR_CUDA(cudaEventCreate(&e));
    struct EvFree {
        cudaEvent_t *e;
        ~EvFree() { for (int k = 0; k < 4; ++k) cudaEventDestroy(e[k]); }
    } evfree{ev};
    auto phase_ms = [&](int a, int b) {
        float ms = 0;
        PR_CUDA(cudaEventSynchronize(ev[b]));
        PR_CUDA(cudaEventElapsedTime(&ms, ev[a], ev[b]));
        return (double)ms;
    };
    for (int l = 0;; ++l) {
        Level &L = h.lev[l];
        int n = L.n;
        L.dinv = dmalloc<double>(n, s);
        if (prm.precision >= 1) L.dinv32 = dmalloc<float>(n, s);
        k_dinv<<<blocks_for(n, BS), BS, 0, s>>>(n, L.rowptr, L.col, L.val, L.dinv, L.dinv32);
        PR_LAUNCH();
        L.cf = dmalloc<int8_t>(n, s);
        L.pmap = dmalloc<int>(n, s);
        // per-matrix stats of this level
        PR_CUDA(cudaMemsetAsync(dnnz, 0, sizeof(long long) * ND, s));
        k_rowlen_dir<<<blocks_for(n, BS), BS, 0, s>>>(n, L.rowptr, L.rowdir, (unsigned long long *)dnnz);
        PR_LAUNCH();
        std::vector<long long> nnzd(ND);
        d2h(nnzd.data(), dnnz, ND, s);
        L.nnzdir.assign(ND, 0);
        for (int d = 0; d < ND; ++d) L.nnzdir[d] = (int)nnzd[d];
        L.ncdir.assign(ND, 0);
        L.nnzZdir.assign(ND, 0);
        L.singular.assign(ND, 0);
        L.coarsest.assign(ND, 0);
        std::vector<char> work(ND, 0);
        bool any = false;
        for (int d = 0; d < ND; ++d) {
            if (L.nrows[d] == 0) continue;
            bool last = L.nrows[d] <= prm.max_coarse || l >= prm.max_levels - 1 || l >= 63;
            L.coarsest[d] = last;
            work[d] = !last;
            any |= !last;
        }
        if (!any) {
            k_fill_int8<<<blocks_for(n, BS), BS, 0, s>>>(n, L.cf, CF_COARSEST);
            PR_LAUNCH();
            k_fill_int<<<blocks_for(n, BS), BS, 0, s>>>(n, L.pmap, -1);
            PR_LAUNCH();
            finish_segments(h, L);
            break;
        }
        PR_CUDA(cudaMemcpyAsync(dwork, work.data(), ND, cudaMemcpyHostToDevice, s));
        PR_CUDA(cudaEventRecord(ev[0], s));
        long long nnz = L.nnz;
        uint8_t *S = dmalloc<uint8_t>(nnz, s);
        k_strength<<<blocks_for(n, BS), BS, 0, s>>>(n, L.rowptr, L.col, L.val, L.rowdir, dwork, prm.theta,
                                                    prm.eps_R, S);
        PR_LAUNCH();
        unsigned *lam = dmalloc<unsigned>(n, s);
        PR_CUDA(cudaMemsetAsync(lam, 0, sizeof(unsigned) * n, s));
        k_lambda<<<blocks_for(n, BS), BS, 0, s>>>(n, L.rowptr, L.col, S, lam);
        PR_LAUNCH();
        uint64_t *key = dmalloc<uint64_t>(n, s);
        int8_t *st0 = dmalloc<int8_t>(n, s), *st1 = dmalloc<int8_t>(n, s);
        int *notmax = dmalloc<int>(n, s);
        PR_CUDA(cudaMemsetAsync(notmax, 0, sizeof(int) * n, s));
        PR_CUDA(cudaMemsetAsync(d_count, 0, sizeof(int), s));
        k_pmis_init<<<blocks_for(n, BS), BS, 0, s>>>(n, L.rowdir, dwork, L.d_row0, lam, l,
                                                     (unsigned long long)prm.seed, key, st0, d_count);
        PR_LAUNCH();
        int und = 0;
        d2h(&und, d_count, 1, s);
        // rounds in groups of PMIS_GROUP between host reads: a round after the last
        // undecided point is gone changes nothing, and the per-round counts give the
        // exact round count
        constexpr int PMIS_GROUP = 4;
        int *rcount = dmalloc<int>(PMIS_GROUP, s);
        int round = 0;
        while (und > 0) {
            PR_REQUIRE(round < 10000, PAIR_ERR_DEVICE, "PMIS did not terminate");
            PR_CUDA(cudaMemsetAsync(rcount, 0, sizeof(int) * PMIS_GROUP, s));
            for (int g = 0; g < PMIS_GROUP; ++g) {
                const int rd = round + 1 + g;
                k_pmis_mark<<<blocks_for(n, BS), BS, 0, s>>>(n, L.rowptr, L.col, S, key, st0, notmax, rd);
                PR_LAUNCH();
                k_pmis_update<<<blocks_for(n, BS), BS, 0, s>>>(n, L.rowptr, L.col, S, st0, st1, notmax, rd,
                                                               rcount + g);
                PR_LAUNCH();
                std::swap(st0, st1);
            }
            int cnt[PMIS_GROUP];
            d2h(cnt, rcount, PMIS_GROUP, s);
            int g = 0;
            while (g < PMIS_GROUP - 1 && cnt[g] > 0) ++g;
            round += g + 1;
            und = cnt[g];
        }
        dfree(rcount, s);
        L.pmis_rounds = round;
        PR_CUDA(cudaEventRecord(ev[1], s));
        PR_CUDA(cudaMemsetAsync(dnc, 0, sizeof(int) * ND, s));
        k_count_c<<<blocks_for(n, BS), BS, 0, s>>>(n, L.rowdir, st0, dnc);
        PR_LAUNCH();
        std::vector<int> ncd(ND);
        d2h(ncd.data(), dnc, ND, s);
        std::vector<char> cont(ND, 0);
        bool anycont = false;
        for (int d = 0; d < ND; ++d) {
            if (!work[d]) continue;
            int nc_ = ncd[d];
            bool stall = nc_ == 0 || (double)nc_ >= 0.9 * (double)L.nrows[d];
            if (stall) L.coarsest[d] = 1;
            else { cont[d] = 1; anycont = true; L.ncdir[d] = nc_; }
        }
        PR_CUDA(cudaMemcpyAsync(dcont, cont.data(), ND, cudaMemcpyHostToDevice, s));
        int *isC = dmalloc<int>(n, s);
        int *cidx = dmalloc<int>(n + 1, s);
        k_cf_final<<<blocks_for(n, BS), BS, 0, s>>>(n, L.rowdir, dcont, st0, L.cf, isC);
        PR_LAUNCH();
        long long nct = scan_exclusive(isC, cidx, n, s);
        dfree(isC, s); dfree(lam, s); dfree(key, s); dfree(st0, s); dfree(st1, s); dfree(notmax, s);
        if (!anycont || nct == 0) {
            k_fill_int<<<blocks_for(n, BS), BS, 0, s>>>(n, L.pmap, -1);
            PR_LAUNCH();
            dfree(S, s); dfree(cidx, s);
            finish_segments(h, L);
            break;
        }
        int nc = (int)nct;
        L.nc = nc;
        L.cpts = dmalloc<int>(nc, s);
        k_cpts<<<blocks_for(n, BS), BS, 0, s>>>(n, L.cf, cidx, L.cpts);
        PR_LAUNCH();
        k_pmap<<<blocks_for(n, BS), BS, 0, s>>>(n, L.rowptr, L.col, L.val, S, L.cf, cidx, L.pmap);
        PR_LAUNCH();
        dfree(cidx, s);

        // ---- lAIR -----------------------------------------------------------
        const int rdist = prm.nair ? 2 : prm.distance;   // nAIR degree 1 uses the distance-2 pattern
        int *ncand = dmalloc<int>(nc, s);
        k_lair_ncand<<<blocks_for(nc, BS), BS, 0, s>>>(nc, L.cpts, L.rowptr, L.col, S, L.cf, rdist, ncand);
        PR_LAUNCH();
        int *candptr = dmalloc<int>(nc + 1, s);
        long long ncandt = scan_exclusive(ncand, candptr, nc, s);
        int *cand = dmalloc<int>(ncandt, s);
        int *npat = ncand;   // reuse
        k_lair_pattern<<<blocks_for(nc, BS), BS, 0, s>>>(nc, L.cpts, L.rowptr, L.col, S, L.cf, rdist, candptr, cand,
                                                         npat);
        PR_LAUNCH();
        int *zr = dmalloc<int>(nc + 1, s);
        long long nz = scan_exclusive(npat, zr, nc, s);
        int *zc = dmalloc<int>(nz, s);
        double *zv = dmalloc<double>(nz, s);
        int *keep = dmalloc<int>(nc, s);
        int *dsing = dmalloc<int>(ND, s);
        PR_CUDA(cudaMemsetAsync(dsing, 0, sizeof(int) * ND, s));
        if (prm.nair) {
            k_nair<<<blocks_for(nc, 128), 128, 0, s>>>(nc, L.cpts, L.rowptr, L.col, L.val, S, L.cf, L.dinv, candptr,
                                                       cand, npat, zr, zc, zv, keep, dsing, L.rowdir, prm.phi_R);
            PR_LAUNCH();
        } else {
            // rows binned by system size; shared memory per warp sized to the bin
            int8_t *ccls = dmalloc<int8_t>(nc, s);
            k_lair_classes<<<blocks_for(nc, BS), BS, 0, s>>>(nc, npat, ccls);
            PR_LAUNCH();
            int hc[LAIR_CLASSES], hstart[LAIR_CLASSES];
            int *list = dmalloc<int>(nc, s);
            partition_by_class(ccls, nc, LAIR_CLASSES, list, hstart, hc, s);
            dfree(ccls, s);
            // n <= 8: a thread per system; 9..24 unknowns: 32 / G systems per warp (G = 8
            // lanes each up to 16 unknowns, 16 lanes up to 24); larger: a warp per system
            auto thread_bin = [&](int c, auto kern, int nm) {
                if (!hc[c]) return;
                size_t sm = (size_t)64 * (nm * nm + 3 * nm) * sizeof(double);
                if (sm > 48 * 1024) allow_max_dyn_smem(kern);
                kern<<<blocks_for(hc[c], 64), 64, sm, s>>>(hc[c], list + hstart[c], L.cpts, L.rowptr, L.col, L.val,
                                                           candptr, cand, npat, zr, zc, zv, keep, dsing, L.rowdir,
                                                           prm.phi_R);
                PR_LAUNCH();
            };
            const int cls_n[LAIR_CLASSES] = {4, 6, 8, 12, 16, 24, 32, 48, 64, 0};
            int smem_optin = 0;
            {
                int dev = 0;
                PR_CUDA(cudaGetDevice(&dev));
                PR_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
            }
            auto warp_bin = [&](int c, auto kern, int G) {
                if (!hc[c]) return;
                const int nm = cls_n[c], spw = 32 / G;
                size_t per = ((size_t)nm * nm + 4 * nm) * sizeof(double) * spw;   // per warp
                // as many warps per block as the shared memory of one block holds (the
                // solves are latency- and FP64-bound, so resident warps decide)
                int wpb = (int)std::max<size_t>(1, std::min<size_t>(32, (size_t)smem_optin / per));
                cudaFuncAttributes fa;   // and no more threads than its registers allow
                PR_CUDA(cudaFuncGetAttributes(&fa, kern));
                wpb = std::max(1, std::min(wpb, fa.maxThreadsPerBlock / 32));
                size_t sm = per * wpb;
                unsigned grid = std::min<unsigned>(blocks_for(hc[c], wpb * spw), 152u * 64u);
                if (sm > 48 * 1024) allow_max_dyn_smem(kern);
                kern<<<grid, 32 * wpb, sm, s>>>(hc[c], list + hstart[c], L.cpts, L.rowptr, L.col, L.val, candptr,
                                                cand, npat, zr, zc, zv, keep, dsing, L.rowdir, prm.phi_R, nm, nullptr,
                                                nullptr);
                PR_LAUNCH();
            };
            thread_bin(0, k_lair_solve_thread<4>, 4);
            thread_bin(1, k_lair_solve_thread<6>, 6);
            thread_bin(2, k_lair_solve_thread<8>, 8);
            warp_bin(3, k_lair_solve<8>, 8);
            warp_bin(4, k_lair_solve<8>, 8);
            warp_bin(5, k_lair_solve<16>, 16);
            for (int c = 6; c < LAIR_BIG; ++c) warp_bin(c, k_lair_solve<32>, 32);
            int nbig = hc[LAIR_BIG];
            if (nbig > 0) {
                long long *goff = dmalloc<long long>(nbig + 1, s);
                k_big_rows<<<blocks_for(nbig, BS), BS, 0, s>>>(nbig, list + hstart[LAIR_BIG], npat, goff);
                PR_LAUNCH();
                const long long gtot = scan_exclusive_ll(goff, nbig, s);
                double *gbuf = dmalloc<double>(gtot, s);
                k_lair_solve<32><<<std::min<unsigned>(nbig, 152u * 16u), 32, 0, s>>>(
                    nbig, list + hstart[LAIR_BIG], L.cpts, L.rowptr, L.col, L.val, candptr, cand, npat, zr, zc, zv, keep,
                    dsing, L.rowdir, prm.phi_R, 0, goff, gbuf);
                PR_LAUNCH();
                dfree(gbuf, s); dfree(goff, s);
            }
            dfree(list, s);
        }
        d2h(L.singular.data(), dsing, ND, s);
        dfree(dsing, s);
        int *zr2 = dmalloc<int>(nc + 1, s);
        long long nz2 = scan_exclusive(keep, zr2, nc, s);
        if (nz2 != nz) {
            int *zc2 = dmalloc<int>(nz2, s);
            double *zv2 = dmalloc<double>(nz2, s);
            k_compact_rows<<<blocks_for(8LL * nc, BS), BS, 0, s>>>(nc, zr, zr2, zc, zv, zc2, zv2);
            PR_LAUNCH();
            dfree(zc, s); dfree(zv, s); dfree(zr, s);
            zc = zc2; zv = zv2;
        } else {
            dfree(zr, s);
        }
        L.zrowptr = zr2; L.zcol = zc; L.zval = zv; L.nnzZ = nz2;
        dfree(keep, s); dfree(cand, s); dfree(candptr, s); dfree(ncand, s);
        dfree(S, s);

        PR_CUDA(cudaEventRecord(ev[2], s));
        // ---- RAP ------------------------------------------------------------
        int *aplen = dmalloc<int>(n, s);
        int *apcol = dmalloc<int>(nnz, s);
        double *apval = dmalloc<double>(nnz, s);
        k_ap<<<blocks_for(n, BS), BS, 0, s>>>(n, L.rowptr, L.col, L.val, L.pmap, L.cf, aplen, apcol, apval);
        PR_LAUNCH();
        int *U = dmalloc<int>(nc, s);
        k_rap_bound<<<blocks_for(nc, BS), BS, 0, s>>>(nc, L.cpts, L.zrowptr, L.zcol, aplen, U);
        PR_LAUNCH();
        int *uptr = dmalloc<int>(nc + 1, s);
        long long ut = scan_exclusive(U, uptr, nc, s);
        int *ucol = dmalloc<int>(ut, s);
        double *uval = dmalloc<double>(ut, s);
        int *cnt = dmalloc<int>(nc, s);
        {
            // rows binned by their bound U: tables of 128 / 512 / 2048 slots in
            // shared memory, larger rows in global scratch
            int8_t *rcls = dmalloc<int8_t>(nc, s);
            k_rap_classes<<<blocks_for(nc, BS), BS, 0, s>>>(nc, U, rcls);
            PR_LAUNCH();
            int hb[4], bstart[4];
            int *rlist = dmalloc<int>(nc, s);
            partition_by_class(rcls, nc, 4, rlist, bstart, hb, s);
            dfree(rcls, s);
            const int caps[3] = {128, 512, 2048};
            int filt = prm.phi_A > 0.0 ? 1 : 0;
            PR_CUDA(cudaMemsetAsync(d_count, 0, sizeof(int), s));
            for (int c = 0; c < 3; ++c) {
                if (!hb[c]) continue;
                int hcap = caps[c];
                bool grp = c == 0;   // small rows: 8 lanes per row, 4 rows per warp
                int spw = grp ? 4 : 1;
                int wpb = std::max(1, std::min(16, (200 * 1024) / (hcap * 12 * spw)));
                size_t sm = (size_t)hcap * wpb * spw * (sizeof(double) + sizeof(int));
                unsigned grid = std::min<unsigned>(blocks_for(hb[c], wpb * spw), 152u * 32u);
                if (grp) {
                    allow_max_dyn_smem(k_rap<8, false>);
                    k_rap<8, false><<<grid, 32 * wpb, sm, s>>>(hb[c], rlist + bstart[c], L.cpts, L.zrowptr, L.zcol,
                                                               L.zval, L.rowptr, aplen, apcol, apval, uptr, U, filt,
                                                               prm.phi_A, cnt, ucol, uval, hcap, nullptr, nullptr,
                                                               nullptr, d_count, h.d_err);
                } else {
                    allow_max_dyn_smem(k_rap<32, false>);
                    k_rap<32, false><<<grid, 32 * wpb, sm, s>>>(hb[c], rlist + bstart[c], L.cpts, L.zrowptr, L.zcol,
                                                                L.zval, L.rowptr, aplen, apcol, apval, uptr, U, filt,
                                                                prm.phi_A, cnt, ucol, uval, hcap, nullptr, nullptr,
                                                                nullptr, d_count, h.d_err);
                }
                PR_LAUNCH();
            }
            int nover = hb[3];
            if (nover > 0) {
                int *list = rlist + bstart[3];
                long long *capw = dmalloc<long long>(nover + 1, s);
                k_overflow_caps<<<blocks_for(nover, BS), BS, 0, s>>>(nover, list, U, capw);
                PR_LAUNCH();
                const long long gtot = scan_exclusive_ll(capw, nover, s);
                int *gk = dmalloc<int>(gtot, s);
                double *gv = dmalloc<double>(gtot, s);
                k_rap<32, true><<<std::min<unsigned>(nover, 152u * 16u), 32, 0, s>>>(
                    nover, list, L.cpts, L.zrowptr, L.zcol, L.zval, L.rowptr, aplen, apcol, apval, uptr, U, filt,
                    prm.phi_A, cnt, ucol, uval, 0, capw, gk, gv, d_count, h.d_err);
                PR_LAUNCH();
                dfree(gk, s); dfree(gv, s); dfree(capw, s);
            }
            int nrej = 0;
            d2h(&nrej, d_count, 1, s);
            PR_REQUIRE(nrej == 0, PAIR_ERR_DEVICE, "RAP row exceeded its table bin");
            dfree(rlist, s);
        }
        Level C;
        C.n = nc;
        C.rowptr = dmalloc<int>(nc + 1, s);
        C.nnz = scan_exclusive(cnt, C.rowptr, nc, s);
        C.col = dmalloc<int>(C.nnz, s);
        C.val = dmalloc<double>(C.nnz, s);
        k_compact_rows<<<blocks_for(8LL * nc, BS), BS, 0, s>>>(nc, uptr, C.rowptr, ucol, uval, C.col, C.val);
        PR_LAUNCH();
        dfree(ucol, s); dfree(uval, s); dfree(uptr, s); dfree(U, s); dfree(cnt, s);
        dfree(aplen, s); dfree(apcol, s); dfree(apval, s);
        C.rowdir = dmalloc<int>(nc, s);
        k_gather_rowdir<<<blocks_for(nc, BS), BS, 0, s>>>(nc, L.cpts, L.rowdir, C.rowdir);
        PR_LAUNCH();
        // nnz of Z per matrix (host, from the Z row pointer at the coarse row ranges)
        {
            C.row0.assign(ND, 0);
            C.nrows.assign(ND, 0);
            std::vector<int> bidx(ND + 1);
            int r = 0;
            for (int d = 0; d < ND; ++d) {
                C.row0[d] = r;
                C.nrows[d] = cont[d] ? L.ncdir[d] : 0;
                bidx[d] = r;
                r += C.nrows[d];
            }
            bidx[ND] = r;
            int *didx = dmalloc<int>(ND + 1, s), *dz = dmalloc<int>(ND + 1, s);
            PR_CUDA(cudaMemcpyAsync(didx, bidx.data(), sizeof(int) * (ND + 1), cudaMemcpyHostToDevice, s));
            k_gather_int<<<blocks_for(ND + 1, BS), BS, 0, s>>>(ND + 1, L.zrowptr, didx, dz);
            PR_LAUNCH();
            std::vector<int> zb(ND + 1);
            d2h(zb.data(), dz, ND + 1, s);   // also orders the host copy of bidx before it is freed
            for (int d = 0; d < ND; ++d) L.nnzZdir[d] = zb[d + 1] - zb[d];
            dfree(didx, s);
            dfree(dz, s);
        }
        C.d_row0 = dmalloc<int>(ND, s);
        PR_CUDA(cudaMemcpyAsync(C.d_row0, C.row0.data(), sizeof(int) * ND, cudaMemcpyHostToDevice, s));
        PR_CUDA(cudaEventRecord(ev[3], s));
        h.t_phase[0] += phase_ms(0, 1);
        h.t_phase[1] += phase_ms(1, 2);
        h.t_phase[2] += phase_ms(2, 3);
        finish_segments(h, L);
        h.lev.push_back(C);
    }
    int err = 0;
    d2h(&err, h.d_err, 1, s);
    dfree(d_count, s); dfree(dwork, s); dfree(dcont, s); dfree(dnc, s); dfree(dnnz, s);
    PR_REQUIRE(err == 0, PAIR_ERR_DEVICE, "setup kernel reported device error bits " + std::to_string(err));
    // V-cycle storage in the cycle precision: the CF split with SELL copies of the F
    // and C rows (the block-form level 0 relaxes without them) and of Z
    for (size_t l = 0; l < h.lev.size(); ++l) {
        Level &L = h.lev[l];
        build_split(h, L, !(l == 0 && h.bsr0));
        if (L.nc > 0) {
            build_sell(h, L.sZ, nullptr, L.nc, L.zrowptr, L.zcol, L.zval);
            sell_compress_cols(h, L.sZ, L.cpts);   // offsets from each coarse point's fine row
        }
    }
    PR_CUDA(cudaStreamSynchronize(s));
}

}  // namespace pr
