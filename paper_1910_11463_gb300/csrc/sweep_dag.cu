// Exact solve of the block-scaled upwind DG system on any mesh (tetrahedra
// included) by a level-scheduled GPU sweep (Sec. 1.1: the transport sweep;
// Sec. 6 compares pAIR with sweeps).
//
// After block-inverse scaling (Sec. 1.3) every diagonal block is the identity,
// so an element whose upwind neighbours are known follows from
//     x_e = b_e - sum_{f upwind of e} A_ef x_f.
// The plan groups elements into levels, level(e) = 1 + max level of e's upwind
// elements, and one launch per level solves all of its elements at once.  On a
// jittered tetrahedral mesh the element graph can be cyclic (on the workloads
// here: faces nearly parallel to Omega, where the rounded Omega.n comes out
// negative on both sides); each cycle is found as a small strongly connected
// component and solved as one dense block by LU with partial pivoting.
//
// Plan, on the device (the host reads one counter row per SD_PASSES levels):
//  1. deps: the distinct elements each element's rows reference (at most the
//     element's face count);
//  2. level passes (Kahn's algorithm): an unassigned element joins level k when
//     every upwind element has a level below k;
//  3. when a direction assigns nothing at level k but still has elements left,
//     its source components -- sets closed under unassigned upwind elements
//     that are strongly connected, at most SD_MAXE elements -- are found by a
//     bounded upwind search from every unassigned element and join level k;
//  4. per level, a list of the single elements and a range of the component
//     table.
// Solve: per level one launch over its single elements (nb threads per element:
// b minus the upwind products in stored order, separate multiply and subtract,
// so the result is the same bits as a sequential sweep) and, where the level
// has components, one launch over them (one CTA each, dense LU in shared
// memory).  Every launch uses programmatic dependent launch; the SI driver
// captures the sequence into a CUDA graph.
#include "common.cuh"

#include <algorithm>
#include <array>
#include <climits>
#include <memory>

namespace pr {

namespace {

constexpr int SD_BS = 256;
constexpr int SD_PASSES = 16;      // level passes per host read
constexpr int SD_MAXK = 32;        // unknowns of one cyclic component
constexpr int SD_COMP_CAP = 1 << 16;

// distinct elements referenced by the rows of element g (first appearance order)
__global__ void k_sd_deps(long long Eb, int nb, int maxd, const int *rowptr, const int *col, int *deps, int *ndep,
                          int *err) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= Eb) return;
    int k = 0;
    int *dg = deps + g * maxd;
    for (long long r = g * nb; r < (g + 1) * nb; ++r)
        for (int p = rowptr[r]; p < rowptr[r + 1]; ++p) {
            const int c = col[p];
            if (c < 0 || (long long)c >= Eb * nb) { atomicOr(err, DERR_BOUNDS); ndep[g] = k; return; }
            const int u = c / nb;
            if (u == g) continue;
            bool seen = false;
            for (int i = 0; i < k; ++i) seen |= dg[i] == u;
            if (seen) continue;
            if (k == maxd) { atomicOr(err, DERR_SWEEP); ndep[g] = k; return; }
            dg[k++] = u;
        }
    ndep[g] = k;
}

// level pass k: an unassigned element whose upwind elements all have levels < k
// joins level k.  A concurrent write of level k to an upwind element reads as
// -1 or k, and both keep this element out, so the pass is race-free.
__global__ void k_sd_pass(long long Eb, long long E, int k, int maxd, const int *deps, const int *ndep, int *level,
                          int *cnt) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= Eb || level[g] >= 0) return;
    const int *dg = deps + g * maxd;
    const int nd = ndep[g];
    for (int i = 0; i < nd; ++i) {
        const int l = level[dg[i]];
        if (l < 0 || l >= k) return;
    }
    level[g] = k;
    atomicAdd(&cnt[g / E], 1);
}

// upwind closure of g over unassigned elements, breadth first; 0 when it has
// more than SD_MAXE elements
__device__ int sd_closure(int g, int maxd, const int *deps, const int *ndep, const int *level, int *B) {
    int sz = 1;
    B[0] = g;
    for (int i = 0; i < sz; ++i) {
        const int v = B[i];
        const int *dv = deps + (long long)v * maxd;
        const int nv = ndep[v];
        for (int j = 0; j < nv; ++j) {
            const int f = dv[j];
            if (level[f] >= 0) continue;
            bool in = false;
            for (int t = 0; t < sz; ++t) in |= B[t] == f;
            if (in) continue;
            if (sz == SD_MAXE) return 0;
            B[sz++] = f;
        }
    }
    return sz;
}

__global__ void k_sd_find(long long Eb, long long E, int maxd, const int *deps, const int *ndep, const int *level,
                          const int8_t *stuck, int *csz, int *crep) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= Eb) return;
    csz[g] = 0;
    if (level[g] >= 0 || !stuck[g / E]) return;
    int B[SD_MAXE];
    const int sz = sd_closure((int)g, maxd, deps, ndep, level, B);
    int rep = B[0];
    for (int t = 1; t < sz; ++t) rep = min(rep, B[t]);
    csz[g] = sz;
    crep[g] = rep;
}

// g lies in a source component when every element of its closure has the same
// closure (then each reaches every other upwind, and nothing unassigned lies
// upwind of the set); the smallest element records the component, its members
// in ascending order
__global__ void k_sd_mark(long long Eb, int nb, int maxd, const int *deps, const int *ndep, const int *level,
                          const int *csz, const int *crep, int8_t *insrc, int *comp, int *compn, int *ncomp,
                          int *err) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= Eb) return;
    insrc[g] = 0;
    const int sz = csz[g];
    if (sz == 0) return;
    int B[SD_MAXE];
    sd_closure((int)g, maxd, deps, ndep, level, B);
    for (int t = 0; t < sz; ++t)
        if (csz[B[t]] != sz || crep[B[t]] != crep[g]) return;
    if (sz * nb > SD_MAXK) { atomicOr(err, DERR_SWEEP); return; }
    insrc[g] = 1;
    if (crep[g] != g) return;
    for (int i = 1; i < sz; ++i)   // unknowns in ascending element order
        for (int j = i; j > 0 && B[j - 1] > B[j]; --j) { const int t = B[j]; B[j] = B[j - 1]; B[j - 1] = t; }
    const int c = atomicAdd(ncomp, 1);
    if (c >= SD_COMP_CAP) { atomicOr(err, DERR_SWEEP); return; }
    for (int t = 0; t < sz; ++t) comp[(long long)c * SD_MAXE + t] = B[t];
    compn[c] = sz;
}

__global__ void k_sd_commit(long long Eb, long long E, int k, const int8_t *insrc, int *level, int8_t *role,
                            int *cnt) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= Eb || !insrc[g]) return;
    level[g] = k;
    role[g] = 1;
    atomicAdd(&cnt[g / E], 1);
}

__global__ void k_sd_count(long long Eb, const int *level, const int8_t *role, int *lcnt) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= Eb || role[g]) return;
    atomicAdd(&lcnt[level[g]], 1);
}

__global__ void k_sd_scatter(long long Eb, const int *level, const int8_t *role, const long long *loff, int *lfill,
                             int *list) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= Eb || role[g]) return;
    const int l = level[g];
    list[loff[l] + atomicAdd(&lfill[l], 1)] = (int)g;
}

// one level's single elements: x_r = b_r - sum over the row's upwind entries
// (stored order; this file is compiled without contraction into FMA)
__global__ void __launch_bounds__(SD_BS) k_sd_level(int nb, const int *list, int count, const int *rowptr,
                                                    const int *col, const double *val, const double *b, double *x) {
    pdl_begin();
    const long long t = (long long)blockIdx.x * SD_BS + threadIdx.x;
    const long long i = t / nb;
    if (i >= count) return;
    const int a = (int)(t - i * nb);
    const long long g = list[i];
    const long long r = g * nb + a;
    double s = b[r];
    for (int p = rowptr[r]; p < rowptr[r + 1]; ++p) {
        const int c = col[p];
        if (c / nb == g) continue;
        s = s - val[p] * x[c];
    }
    x[r] = s;
}

// one cyclic component per CTA, solved by thread 0: the component's rows with
// the known upwind values moved to the right-hand side, then LU with partial
// pivoting (first largest |pivot|, multipliers a_rk * (1 / a_kk), fma updates)
// and substitution with y_k * (1 / u_kk)
__global__ void k_sd_comp(int nb, const int *comp, const int *compn, const int *rowptr, const int *col,
                          const double *val, const double *b, double *x, int *err) {
    pdl_begin();
    __shared__ double A[SD_MAXK * SD_MAXK];
    __shared__ double y[SD_MAXK];
    __shared__ int piv[SD_MAXK];
    if (threadIdx.x != 0) return;
    const int *mem = comp + (long long)blockIdx.x * SD_MAXE;
    const int k = compn[blockIdx.x];
    const int m = k * nb;
    for (int i = 0; i < m * m; ++i) A[i] = 0.0;
    for (int i = 0; i < k; ++i)
        for (int a = 0; a < nb; ++a) {
            const long long r = (long long)mem[i] * nb + a;
            const int rr = i * nb + a;
            double s = b[r];
            for (int p = rowptr[r]; p < rowptr[r + 1]; ++p) {
                const int c = col[p], e = c / nb;
                int pe = -1;
                for (int j = 0; j < k; ++j)
                    if (mem[j] == e) pe = j;
                if (pe >= 0) A[rr * m + pe * nb + (c - e * nb)] = val[p];
                else s = s - val[p] * x[c];
            }
            y[rr] = s;
        }
    for (int q = 0; q < m; ++q) {
        int p = q;
        double mx = fabs(A[q * m + q]);
        for (int r = q + 1; r < m; ++r) {
            const double v = fabs(A[r * m + q]);
            if (v > mx) { mx = v; p = r; }
        }
        piv[q] = p;
        if (!(mx > 0.0)) {
            atomicOr(err, DERR_SWEEP);
            for (int i = 0; i < k; ++i)
                for (int a = 0; a < nb; ++a) x[(long long)mem[i] * nb + a] = nan("");
            return;
        }
        if (p != q)
            for (int c = 0; c < m; ++c) { const double t = A[q * m + c]; A[q * m + c] = A[p * m + c]; A[p * m + c] = t; }
        const double rd = 1.0 / A[q * m + q];
        for (int r = q + 1; r < m; ++r) {
            const double l = A[r * m + q] * rd;
            A[r * m + q] = l;
            for (int c = q + 1; c < m; ++c) A[r * m + c] = fma(-l, A[q * m + c], A[r * m + c]);
        }
    }
    for (int q = 0; q < m; ++q)
        if (piv[q] != q) { const double t = y[q]; y[q] = y[piv[q]]; y[piv[q]] = t; }
    for (int q = 0; q < m; ++q)
        for (int r = q + 1; r < m; ++r) y[r] = fma(-A[r * m + q], y[q], y[r]);
    for (int q = m - 1; q >= 0; --q) {
        y[q] = y[q] * (1.0 / A[q * m + q]);
        for (int r = 0; r < q; ++r) y[r] = fma(-A[r * m + q], y[q], y[r]);
    }
    for (int i = 0; i < k; ++i)
        for (int a = 0; a < nb; ++a) x[(long long)mem[i] * nb + a] = y[i * nb + a];
}

int read_err(const int *d_err, cudaStream_t s) {
    int e = 0;
    PR_CUDA(cudaMemcpyAsync(&e, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    PR_CUDA(cudaStreamSynchronize(s));
    return e;
}

}  // namespace

void SweepPlan::release(cudaStream_t s) {
    dfree(list, s);
    dfree(comp, s);
    dfree(compn, s);
    list = comp = compn = nullptr;
}

SweepPlan *sweep_plan_build(int nd, long long N, int nb, const int *rowptr, const int *col, int *d_err,
                            cudaStream_t s) {
    PR_REQUIRE(nb == 4 || nb == 8, PAIR_ERR_ARG, "GPU sweep: 4 or 8 DOFs per element");
    PR_REQUIRE(N % nb == 0 && nd >= 1, PAIR_ERR_ARG, "GPU sweep: rows are not whole elements");
    const long long E = N / nb, Eb = E * nd;
    PR_REQUIRE(Eb * nb < 0x7fffffffLL, PAIR_ERR_UNSUPPORTED, "GPU sweep: more than 2^31 rows");
    const int maxd = nb == 8 ? 6 : 4;   // faces of a hexahedron / tetrahedron
    const unsigned gb = blocks_for(Eb, SD_BS);
    std::vector<void *> tmp;
    auto alloc = [&](size_t bytes) { void *p = dmalloc<char>(bytes, s); tmp.push_back(p); return p; };
    struct Free {
        std::vector<void *> *t;
        cudaStream_t s;
        ~Free() { for (void *p : *t) dfree(p, s); }
    } fr{&tmp, s};
    auto plan = std::make_unique<SweepPlan>();
    struct Release {   // device arrays of a plan that is not handed out
        std::unique_ptr<SweepPlan> *p;
        cudaStream_t s;
        ~Release() { if (*p) (*p)->release(s); }
    } rel{&plan, s};
    plan->nb = nb;
    int *deps = (int *)alloc(sizeof(int) * Eb * maxd), *ndep = (int *)alloc(sizeof(int) * Eb);
    int *level = (int *)alloc(sizeof(int) * Eb);
    int8_t *role = (int8_t *)alloc(Eb);
    int *cnt = (int *)alloc(sizeof(int) * SD_PASSES * nd);
    PR_CUDA(cudaMemsetAsync(level, 0xff, sizeof(int) * Eb, s));
    PR_CUDA(cudaMemsetAsync(role, 0, Eb, s));
    k_sd_deps<<<gb, SD_BS, 0, s>>>(Eb, nb, maxd, rowptr, col, deps, ndep, d_err);
    PR_LAUNCH();
    if (int e = read_err(d_err, s))
        fail(e & DERR_BOUNDS ? PAIR_ERR_ARG : PAIR_ERR_UNSUPPORTED,
             e & DERR_BOUNDS ? "GPU sweep: column outside the matrix"
                             : "GPU sweep: an element references more elements than it has faces");
    // component search state, allocated at the first cycle
    int *csz = nullptr, *crep = nullptr, *d_ncomp = nullptr, *ccnt = nullptr;
    int8_t *insrc = nullptr, *stuck = nullptr;
    std::vector<int> hc((size_t)SD_PASSES * nd), cur(nd, 0);
    std::vector<long long> rem(nd, E);
    std::vector<std::array<int, 3>> comp_lv;   // (level, first, end) in the component table
    int ncomp = 0;
    long long left = Eb, passes = 0;
    int k = 0;
    while (left > 0) {
        // every round assigns at least one element (or fails), so this is a safety net only
        PR_REQUIRE(passes <= (long long)SD_PASSES * (Eb + 4), PAIR_ERR_UNSUPPORTED,
                   "GPU sweep: level schedule does not terminate");
        PR_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * SD_PASSES * nd, s));
        for (int p = 0; p < SD_PASSES; ++p) {
            k_sd_pass<<<gb, SD_BS, 0, s>>>(Eb, E, k + p, maxd, deps, ndep, level, cnt + (size_t)p * nd);
            PR_LAUNCH();
        }
        passes += SD_PASSES;
        PR_CUDA(cudaMemcpyAsync(hc.data(), cnt, sizeof(int) * hc.size(), cudaMemcpyDeviceToHost, s));
        PR_CUDA(cudaStreamSynchronize(s));
        std::vector<int> st(nd, -1);
        int jmin = INT_MAX;
        for (int d = 0; d < nd; ++d) {
            for (int p = 0; p < SD_PASSES && rem[d] > 0; ++p) {
                const int L = k + p;
                if (L < cur[d]) continue;   // levels this direction has completed
                const int c = hc[(size_t)p * nd + d];
                if (c == 0) { st[d] = L; break; }
                rem[d] -= c;
                cur[d] = L + 1;
            }
            if (st[d] >= 0) jmin = std::min(jmin, st[d]);
        }
        if (jmin != INT_MAX) {
            // every direction stuck at level jmin: its source components join level jmin
            if (!csz) {
                csz = (int *)alloc(sizeof(int) * Eb);
                crep = (int *)alloc(sizeof(int) * Eb);
                insrc = (int8_t *)alloc(Eb);
                stuck = (int8_t *)alloc(nd);
                d_ncomp = (int *)alloc(sizeof(int));
                ccnt = (int *)alloc(sizeof(int) * nd);
                plan->comp = dmalloc<int>((size_t)SD_COMP_CAP * SD_MAXE, s);
                plan->compn = dmalloc<int>(SD_COMP_CAP, s);
                PR_CUDA(cudaMemsetAsync(d_ncomp, 0, sizeof(int), s));
            }
            std::vector<int8_t> sf(nd);
            for (int d = 0; d < nd; ++d) sf[d] = st[d] == jmin;
            PR_CUDA(cudaMemcpyAsync(stuck, sf.data(), nd, cudaMemcpyHostToDevice, s));
            PR_CUDA(cudaMemsetAsync(ccnt, 0, sizeof(int) * nd, s));
            k_sd_find<<<gb, SD_BS, 0, s>>>(Eb, E, maxd, deps, ndep, level, stuck, csz, crep);
            PR_LAUNCH();
            k_sd_mark<<<gb, SD_BS, 0, s>>>(Eb, nb, maxd, deps, ndep, level, csz, crep, insrc, plan->comp,
                                           plan->compn, d_ncomp, d_err);
            PR_LAUNCH();
            k_sd_commit<<<gb, SD_BS, 0, s>>>(Eb, E, jmin, insrc, level, role, ccnt);
            PR_LAUNCH();
            std::vector<int> hcc(nd);
            int nc = 0;
            PR_CUDA(cudaMemcpyAsync(hcc.data(), ccnt, sizeof(int) * nd, cudaMemcpyDeviceToHost, s));
            PR_CUDA(cudaMemcpyAsync(&nc, d_ncomp, sizeof(int), cudaMemcpyDeviceToHost, s));
            if (read_err(d_err, s))
                fail(PAIR_ERR_UNSUPPORTED, "GPU sweep: more than 65536 cyclic components or a component of more "
                                           "than 32 unknowns");
            for (int d = 0; d < nd; ++d) {
                if (!sf[d]) continue;
                PR_REQUIRE(hcc[d] > 0, PAIR_ERR_UNSUPPORTED,
                           "GPU sweep: a cycle of the upwind graph spans more than 8 elements");
                rem[d] -= hcc[d];
                cur[d] = jmin + 1;
            }
            comp_lv.push_back({jmin, ncomp, nc});
            ncomp = nc;
        }
        left = 0;
        k = INT_MAX;
        for (int d = 0; d < nd; ++d)
            if (rem[d] > 0) { left += rem[d]; k = std::min(k, cur[d]); }
    }
    int nlev = 0;
    for (int d = 0; d < nd; ++d) nlev = std::max(nlev, cur[d]);
    plan->nlev = nlev;
    plan->ncomp = ncomp;
    // single elements level by level
    int *lcnt = (int *)alloc(sizeof(int) * std::max(nlev, 1)), *lfill = (int *)alloc(sizeof(int) * std::max(nlev, 1));
    long long *loff = (long long *)alloc(sizeof(long long) * (nlev + 1));
    PR_CUDA(cudaMemsetAsync(lcnt, 0, sizeof(int) * std::max(nlev, 1), s));
    PR_CUDA(cudaMemsetAsync(lfill, 0, sizeof(int) * std::max(nlev, 1), s));
    k_sd_count<<<gb, SD_BS, 0, s>>>(Eb, level, role, lcnt);
    PR_LAUNCH();
    std::vector<int> hl(std::max(nlev, 1));
    PR_CUDA(cudaMemcpyAsync(hl.data(), lcnt, sizeof(int) * hl.size(), cudaMemcpyDeviceToHost, s));
    PR_CUDA(cudaStreamSynchronize(s));
    plan->off.assign(nlev + 1, 0);
    for (int l = 0; l < nlev; ++l) plan->off[l + 1] = plan->off[l] + hl[l];
    PR_CUDA(cudaMemcpyAsync(loff, plan->off.data(), sizeof(long long) * (nlev + 1), cudaMemcpyHostToDevice, s));
    plan->list = dmalloc<int>(std::max<long long>(plan->off[nlev], 1), s);
    k_sd_scatter<<<gb, SD_BS, 0, s>>>(Eb, level, role, loff, lfill, plan->list);
    PR_LAUNCH();
    plan->comp_off.assign(nlev + 1, 0);
    for (auto &c : comp_lv) plan->comp_off[c[0] + 1] = c[2] - c[1];
    for (int l = 0; l < nlev; ++l) plan->comp_off[l + 1] += plan->comp_off[l];
    PR_CUDA(cudaStreamSynchronize(s));
    return plan.release();
}

void sweep_plan_launch(const SweepPlan &P, const int *rowptr, const int *col, const double *val, const double *b,
                       double *x, int *d_err, cudaStream_t s) {
    for (int l = 0; l < P.nlev; ++l) {
        const long long c = P.off[l + 1] - P.off[l];
        if (c > 0) {
            launch_pdl(k_sd_level, dim3(blocks_for(c * P.nb, SD_BS)), dim3(SD_BS), s, P.nb,
                       (const int *)(P.list + P.off[l]), (int)c, rowptr, col, val, b, x);
            PR_LAUNCH();
        }
        const int c0 = P.comp_off[l], c1 = P.comp_off[l + 1];
        if (c1 > c0) {
            launch_pdl(k_sd_comp, dim3(c1 - c0), dim3(32), s, P.nb, (const int *)(P.comp + (size_t)c0 * SD_MAXE),
                       (const int *)(P.compn + c0), rowptr, col, val, b, x, d_err);
            PR_LAUNCH();
        }
    }
}

void sweep_csr(int n, int nb, const int *rowptr, const int *col, const double *val, const double *b, double *x,
               cudaStream_t s, int *ncomp, int *nlev) {
    int *d_err = dmalloc<int>(1, s);
    struct Free {
        int *e;
        cudaStream_t s;
        SweepPlan *p = nullptr;
        ~Free() {
            if (p) { p->release(s); delete p; }
            dfree(e, s);
        }
    } fr{d_err, s};
    PR_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), s));
    fr.p = sweep_plan_build(1, n, nb, rowptr, col, d_err, s);
    sweep_plan_launch(*fr.p, rowptr, col, val, b, x, d_err, s);
    PR_REQUIRE(read_err(d_err, s) == 0, PAIR_ERR_SINGULAR, "GPU sweep: singular cyclic component");
    if (ncomp) *ncomp = fr.p->ncomp;
    if (nlev) *nlev = fr.p->nlev;
}

}  // namespace pr
