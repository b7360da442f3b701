// AIR solve loop and S_N source iteration (Eq. sn_transport, Eq. angular_quad).
//
// Each SI iteration, for every direction batch:
//   b_m = W_m s + g Gin_m,   s_K = (sigma_s,K phi_K + q_K) / (4 pi),  W = D^{-1} M
//   psi_m = 0; repeat { r = b - A psi (FP64); stop if ||r|| <= tol ||b||;
//                       psi += V(r) }   (V in FP64 or FP32)
//   phi^{n+1} += sum_m w_m psi_m  (FP64, directions in fixed order)
// then ||phi^{n+1} - phi^n|| / ||phi^{n+1}|| closes the iteration.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <initializer_list>
#include <exception>
#include <string>
#include <thread>
#include <utility>

#include "common.cuh"

namespace pr {

namespace {

constexpr int BS = 256;

// isotropic source per DOF: src = (sigma_s phi + q) / (4 pi)
template <int NB>
__global__ void k_src(long long N, const double *sigma_s, const double *q, const double *phi, double *src) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double inv4pi = 1.0 / (4.0 * 3.14159265358979323846);
    const long long e = i / NB;
    src[i] = (sigma_s[e] * phi[i] + q[e]) * inv4pi;
}

// b = W src (+ W q_ang of the direction) (+ g Gin): thread per row of a direction,
// the row of W in 16-byte loads
template <int NB>
__global__ void k_rhs(long long E, int ndir, const double *W, const double *Gin, double g, const double *src,
                      const double *qa, double *b) {
    long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= NB * E * ndir) return;
    long long m = tid / (NB * E);
    long long r = tid % (NB * E);
    long long e = r / NB;
    int a = (int)(r % NB);
    const double2 *w2 = reinterpret_cast<const double2 *>(W + ((m * E + e) * NB + a) * NB);
    double w[NB];
#pragma unroll
    for (int c = 0; c < NB / 2; ++c) {
        const double2 t = __ldcs(w2 + c);
        w[2 * c] = t.x;
        w[2 * c + 1] = t.y;
    }
    const double *se = src + NB * e;
    double acc = 0.0;
    if (qa) {   // angular source of this direction, added to the isotropic one per node
        const double *qm = qa + (m * E + e) * NB;
#pragma unroll
        for (int c = 0; c < NB; ++c) acc += w[c] * (se[c] + qm[c]);
    } else {
#pragma unroll
        for (int c = 0; c < NB; ++c) acc += w[c] * se[c];
    }
    if (Gin) acc += g * Gin[tid];
    b[tid] = acc;
}

// phinew (+)= sum_m w_m x_m over the batch's directions in order; 'overwrite'
// starts the sum from zero instead of the stored value
__global__ void k_phi_acc(long long N, int nd, const double *w, const double *x, double *phinew, int overwrite) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double acc = overwrite ? 0.0 : phinew[i];
    for (int m = 0; m < nd; ++m) acc += w[m] * x[(long long)m * N + i];
    phinew[i] = acc;
}

// phinew = partial_0 + partial_1 + ... + partial_{K-1}, in that order (the partial
// fluxes of concurrently solved direction groups, each N long)
__global__ void k_phi_sum(long long N, int K, const double *partial, double *phinew) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double acc = partial[i];
    for (int k = 1; k < K; ++k) acc += partial[(long long)k * N + i];
    phinew[i] = acc;
}

__global__ void k_diff_partials(long long N, const double *a, const double *b, double *part) {
    __shared__ double sh[2][32];
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double d2 = 0.0, n2 = 0.0;
    if (i < N) {
        double d = a[i] - b[i];
        d2 = d * d;
        n2 = a[i] * a[i];
    }
    for (int o = 16; o > 0; o >>= 1) {
        d2 += __shfl_down_sync(0xffffffffu, d2, o);
        n2 += __shfl_down_sync(0xffffffffu, n2, o);
    }
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { sh[0][w] = d2; sh[1][w] = n2; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0, s1 = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { s0 += sh[0][k]; s1 += sh[1][k]; }
        part[2 * blockIdx.x] = s0;
        part[2 * blockIdx.x + 1] = s1;
    }
}

// one block of DIFF_BS threads: thread t sums partials t, t + DIFF_BS, ... in order,
// then a fixed tree (deterministic)
constexpr int DIFF_BS = 256;
__global__ void k_diff_final(int nb, const double *part, double *out) {
    __shared__ double sh[2][DIFF_BS];
    double s0 = 0, s1 = 0;
    for (int k = threadIdx.x; k < nb; k += DIFF_BS) { s0 += part[2 * k]; s1 += part[2 * k + 1]; }
    sh[0][threadIdx.x] = s0;
    sh[1][threadIdx.x] = s1;
    __syncthreads();
    for (int h = DIFF_BS / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + h];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sqrt(sh[0][0]);
        out[1] = sqrt(sh[1][0]);
    }
}

__global__ void k_fill_dir(int *rowdir, long long N, int ndir) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N * ndir) rowdir[i] = (int)(i / N);
}

// flag |= 1 if any of a[0..n) is NaN or Inf (grid-stride)
__global__ void k_nonfinite(long long n, const double *a, int *flag) {
    int bad = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        bad |= !isfinite(a[i]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

}  // namespace


// ---- instrumentation --------------------------------------------------------------
namespace {

float elapsed_ms(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0;
    PR_CUDA(cudaEventElapsedTime(&ms, a, b));
    return ms;
}

// outer residual (ev[0..1]) of the matrices that took part
void account_outer(Hier &h, const std::vector<char> &part) {
    if (!h.timed) return;
    h.t_res0 += elapsed_ms(h.ev[0], h.ev[1]);
    h.n_res0 += 1;
    double br = 0;
    for (int d = 0; d < h.ndir; ++d)
        if (part[d]) br += h.bytes_res0[d];
    h.gb_res0 += br * 1e-9;
}

// one V-cycle recorded in slot ps: level-0 relaxation and inner residual of the
// matrices that took part, coarse-level relaxation (every matrix of the batch)
void account_cycle(Hier &h, const ProfSlot &ps, const std::vector<char> &part) {
    if (!h.timed) return;
    double bx = 0, b32 = 0;
    for (int d = 0; d < h.ndir; ++d)
        if (part[d]) {
            bx += h.bytes_relax0[d];
            if (!h.bytes_res32.empty()) b32 += h.bytes_res32[d];
        }
    if (ps.lv.size() >= 4) {
        double tl = 0;
        int nl = 0;
        for (size_t l = 1; l + 1 < h.lev.size() && 2 * l + 1 < ps.lv.size(); ++l) {
            if (!h.lev[l].n) continue;
            const float t = elapsed_ms(ps.lv[2 * l], ps.lv[2 * l + 1]);
            tl += t;
            h.t_relaxc_level[std::min<size_t>(l, 8) - 1] += t;
            ++nl;
        }
        // grid-wide coarsest sweeps (levels with a SELL copy of their coarsest rows)
        for (size_t l = 1; l < h.lev.size() && 2 * l + 1 < ps.lvx.size(); ++l) {
            if (h.lev[l].sX.nrows <= 0) continue;
            const float t = elapsed_ms(ps.lvx[2 * l], ps.lvx[2 * l + 1]);
            tl += t;
            h.t_relaxc_level[std::min<size_t>(l, 8) - 1] += t;
            ++nl;
        }
        if (nl) {
            h.t_relaxc += tl;
            h.n_relaxc += 1;
            h.gb_relaxc += h.bytes_relaxc * 1e-9;
        }
    }
    if (ps.lvt.size() >= 4 && h.lev.size() >= 2) {
        double tx = 0;
        for (size_t l = 0; l + 1 < h.lev.size() && 4 * l + 3 < ps.lvt.size(); ++l)
            tx += elapsed_ms(ps.lvt[4 * l], ps.lvt[4 * l + 1]) + elapsed_ms(ps.lvt[4 * l + 2], ps.lvt[4 * l + 3]);
        h.t_xfer += tx;
        h.n_xfer += 1;
        h.gb_xfer += h.bytes_xfer * 1e-9;
    }
    if (ps.relax_timed) {
        h.t_relax0 += elapsed_ms(ps.relax0[0], ps.relax0[1]);
        h.n_relax0 += 1;
        h.gb_relax0 += bx * 1e-9;
    }
    if (ps.res_timed) {
        h.t_res32 += elapsed_ms(ps.res32[0], ps.res32[1]);
        h.n_res32 += 1;
        h.gb_res32 += b32 * 1e-9;
    }
}

template <class F>
cudaGraphExec_t capture(Hier &h, long long &kernels, F &&body) {
    cudaGraph_t g;
    const long long before = g_thread_launches;
    PR_CUDA(cudaStreamBeginCapture(h.stream, cudaStreamCaptureModeThreadLocal));
    try {
        body();
    } catch (...) {
        cudaGraph_t dummy = nullptr;
        cudaStreamEndCapture(h.stream, &dummy);
        if (dummy) cudaGraphDestroy(dummy);
        g_launches -= g_thread_launches - before;
        throw;
    }
    PR_CUDA(cudaStreamEndCapture(h.stream, &g));
    kernels = g_thread_launches - before;
    g_launches -= kernels;   // counted per replay instead
    cudaGraphExec_t ex = nullptr;
    cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    PR_CUDA(e);
    return ex;
}

ProfSlot *slot(Hier &h, int k) { return h.timed && k < (int)h.slots.size() ? &h.slots[k] : nullptr; }

}  // namespace

// One-time capture of [V-cycle correction; residual] for fixed (b, x, tol).
static void ensure_graph(Hier &h, const double *b, double *x, double tol) {
    CycleGraphs &G = h.graphs();
    if (G.graph && G.graph_b == b && G.graph_x == x && G.graph_tol == tol) return;
    if (G.graph) { cudaGraphExecDestroy(G.graph); G.graph = nullptr; }
    G.graph = capture(h, G.graph_kernels, [&] {
        vcycle_correct(h, x, slot(h, 0));
        residual0(h, b, x, tol, true);
    });
    G.graph_b = b;
    G.graph_x = x;
    G.graph_tol = tol;
}

namespace {

// 2^g inner cycles on the slots [2^g - 1, 2^(g+1) - 1): one graph launch, or the
// launches themselves
void run_inner(Hier &h, int g, bool use_graph) {
    const int k = 1 << g;
    if (use_graph) {
        CycleGraphs &G = h.graphs();
        if (!G.gcyc[g])
            G.gcyc[g] = capture(h, G.gcyc_kernels[g], [&] {
                for (int t = 0; t < k; ++t) inner_cycle(h, slot(h, k - 1 + t));
            });
        PR_CUDA(cudaGraphLaunch(G.gcyc[g], h.stream));
        g_launches += G.gcyc_kernels[g];
    } else {
        for (int t = 0; t < k; ++t) inner_cycle(h, slot(h, k - 1 + t));
    }
}

// end of a refinement step: x += d, new outer residual, norms and flags
void run_close(Hier &h, const double *b, double *x, double tol, bool use_graph) {
    if (use_graph) {
        CycleGraphs &G = h.graphs();
        if (!G.gclose || G.gi_b != b || G.gi_x != x || G.gi_tol != tol) {
            if (G.gclose) { cudaGraphExecDestroy(G.gclose); G.gclose = nullptr; }
            G.gclose = capture(h, G.gclose_kernels, [&] {
                fold_delta(h, x);
                residual_outer(h, b, x, tol);
            });
            G.gi_b = b;
            G.gi_x = x;
            G.gi_tol = tol;
        }
        PR_CUDA(cudaGraphLaunch(G.gclose, h.stream));
        g_launches += G.gclose_kernels;
    } else {
        fold_delta(h, x);
        residual_outer(h, b, x, tol);
    }
}

// Iterative refinement with an FP32 inner iteration (Sec. 2.1 solve loop; the
// precision split of the method's FP32-refined form): each step takes the outer
// residual r = b - A x (FP64, or double-float on the hex block form), iterates
// A d = r with FP32 V-cycles and FP32 residuals until every matrix reaches its step
// threshold, then x += d.  The host reads flags and norms once per step; the
// cycles of a step are launched back to back (the count predicted from the
// measured contraction, as graphs of 1, 2, 4 and 8 cycles), and matrices (and, once
// none is left, whole launches) that reached their threshold do no work.
BatchSolve solve_batch_inner(Hier &h, const double *b, double *x, double tol, int maxit, bool use_graph,
                             bool x_zero) {
    cudaStream_t s = h.stream;
    const int nd = h.ndir;
    norms0(h, b, h.bnorm);
    set_all_active(h);
    PR_CUDA(cudaMemsetAsync(h.icount, 0, sizeof(int) * nd, s));
    if (h.dd) dd_load(h, b, x);
    residual_outer(h, b, x, tol, x_zero);
    std::vector<double> r0(nd), rn(nd), bn(nd), inn(nd);
    std::vector<int> act(nd), cnt(nd, 0), cyc(nd, 0);
    PR_CUDA(cudaMemcpyAsync(r0.data(), h.rnorm, sizeof(double) * nd, cudaMemcpyDeviceToHost, s));
    PR_CUDA(cudaMemcpyAsync(bn.data(), h.bnorm, sizeof(double) * nd, cudaMemcpyDeviceToHost, s));
    PR_CUDA(cudaMemcpyAsync(act.data(), h.active, sizeof(int) * nd, cudaMemcpyDeviceToHost, s));
    PR_CUDA(cudaStreamSynchronize(s));
    if (!x_zero) account_outer(h, std::vector<char>(nd, 1));
    for (int d = 0; d < nd; ++d)
        if (!std::isfinite(r0[d]) || !std::isfinite(bn[d])) fail(PAIR_ERR_NAN, "NaN/Inf in right-hand side or residual");
    rn = r0;
    int outer = x_zero ? 0 : 1;   // residuals that read the operator
    bool any = std::any_of(act.begin(), act.end(), [](int a) { return a != 0; });
    while (any) {
        int done = 0;
        for (int d = 0; d < nd; ++d)
            if (act[d]) done = std::max(done, cyc[d]);
        if (done >= maxit) break;
        // cycles this step: enough for the slowest matrix at the measured contraction
        const double rho = h.rho_est > 0 ? h.rho_est : 0.3;
        double want = 1;
        for (int d = 0; d < nd; ++d) {
            if (!act[d] || !(rn[d] > 0)) continue;
            const double target = std::max(INNER_TOL_FRAC * tol * bn[d], INNER_ETA * rn[d]);
            want = std::max(want, std::log(target / rn[d]) / std::log(rho));
        }
        int need = std::min({(int)std::ceil(want + 0.1), INNER_SLOTS, maxit - done});
        need = std::max(need, 1);
        std::vector<int> launched;
        for (int g = INNER_GRAPHS - 1, rem = need; g >= 0; --g)
            if (rem >= (1 << g)) { run_inner(h, g, use_graph); launched.push_back(g); rem -= 1 << g; }
        std::vector<char> was(nd);
        for (int d = 0; d < nd; ++d) was[d] = act[d] != 0;
        run_close(h, b, x, tol, use_graph);
        std::vector<double> rprev = rn;
        PR_CUDA(cudaMemcpyAsync(cnt.data(), h.icount, sizeof(int) * nd, cudaMemcpyDeviceToHost, s));
        PR_CUDA(cudaMemcpyAsync(inn.data(), h.inorm, sizeof(double) * nd, cudaMemcpyDeviceToHost, s));
        PR_CUDA(cudaMemcpyAsync(rn.data(), h.rnorm, sizeof(double) * nd, cudaMemcpyDeviceToHost, s));
        PR_CUDA(cudaMemcpyAsync(act.data(), h.active, sizeof(int) * nd, cudaMemcpyDeviceToHost, s));
        PR_CUDA(cudaStreamSynchronize(s));
        ++outer;
        std::vector<int> sc(nd);   // cycles of this step per matrix (icount accumulates)
        for (int d = 0; d < nd; ++d) sc[d] = cnt[d] - cyc[d];
        // cycle j of the step ran for the matrices with more than j cycles
        if (h.timed) {
            int j = 0;
            for (int g : launched)
                for (int t = 0; t < (1 << g); ++t, ++j) {
                    std::vector<char> part(nd);
                    for (int d = 0; d < nd; ++d) part[d] = was[d] && sc[d] > j;
                    account_cycle(h, h.slots[(1 << g) - 1 + t], part);
                }
            account_outer(h, was);
        }
        double rho_obs = 0;
        for (int d = 0; d < nd; ++d) {
            if (!was[d]) continue;
            cyc[d] += sc[d];
            if (sc[d] > 0 && rprev[d] > 0 && inn[d] > 0)
                rho_obs = std::max(rho_obs, std::pow(inn[d] / rprev[d], 1.0 / sc[d]));
            if (!std::isfinite(rn[d])) fail(PAIR_ERR_NAN, "NaN/Inf in a residual during the AIR solve");
        }
        if (rho_obs > 0) h.rho_est = std::min(0.95, std::max(0.02, rho_obs));
        any = std::any_of(act.begin(), act.end(), [](int a) { return a != 0; });
    }
    if (h.dd) dd_store(h, x);
    PR_CUDA(cudaStreamSynchronize(s));
    BatchSolve out;
    out.outer = outer;
    for (int d = 0; d < nd; ++d) {
        out.iters = std::max(out.iters, cyc[d]);
        out.cycles += cyc[d];
        double rel = bn[d] > 0 ? rn[d] / bn[d] : 0.0;
        out.max_rel = std::max(out.max_rel, rel);
        if (cyc[d] > 0 && r0[d] > 0 && rn[d] > 0) {
            out.rho_sum += std::pow(rn[d] / r0[d], 1.0 / cyc[d]);
            out.rho_cnt++;
        }
    }
    out.converged = !any;
    return out;
}

}  // namespace

// Solves every matrix of the hierarchy from the given x to ||b - A x|| <= tol ||b||.
BatchSolve solve_batch(Hier &h, const double *b, double *x, double tol, int maxit, bool use_graph, bool x_zero) {
    if (h.inner && tol > 0.0) return solve_batch_inner(h, b, x, tol, maxit, use_graph, x_zero);
    cudaStream_t s = h.stream;
    int nd = h.ndir;
    norms0(h, b, h.bnorm);
    set_all_active(h);
    if (h.dd) dd_load(h, b, x);
    residual0(h, b, x, tol, true, x_zero);
    std::vector<double> r0(nd), rn(nd), bn(nd);
    std::vector<int> act(nd), itd(nd, 0);
    PR_CUDA(cudaMemcpyAsync(r0.data(), h.rnorm, sizeof(double) * nd, cudaMemcpyDeviceToHost, s));
    PR_CUDA(cudaMemcpyAsync(bn.data(), h.bnorm, sizeof(double) * nd, cudaMemcpyDeviceToHost, s));
    PR_CUDA(cudaMemcpyAsync(act.data(), h.active, sizeof(int) * nd, cudaMemcpyDeviceToHost, s));
    PR_CUDA(cudaStreamSynchronize(s));
    if (!x_zero) account_outer(h, std::vector<char>(nd, 1));
    for (int d = 0; d < nd; ++d)
        if (!std::isfinite(r0[d]) || !std::isfinite(bn[d])) fail(PAIR_ERR_NAN, "NaN/Inf in right-hand side or residual");
    if (use_graph) ensure_graph(h, b, x, tol);
    int k = 0;
    bool any = std::any_of(act.begin(), act.end(), [](int a) { return a != 0; });
    while (any && k < maxit) {
        if (use_graph) {
            PR_CUDA(cudaGraphLaunch(h.graphs().graph, s));
            g_launches += h.graphs().graph_kernels;
        } else {
            vcycle_correct(h, x, slot(h, 0));
            residual0(h, b, x, tol, true);
        }
        ++k;
        std::vector<char> was(nd);
        for (int d = 0; d < nd; ++d) was[d] = act[d] != 0;
        PR_CUDA(cudaMemcpyAsync(act.data(), h.active, sizeof(int) * nd, cudaMemcpyDeviceToHost, s));
        PR_CUDA(cudaStreamSynchronize(s));
        if (h.timed) {
            account_cycle(h, h.slots[0], was);
            account_outer(h, was);
        }
        any = false;
        for (int d = 0; d < nd; ++d) {
            if (act[d]) { any = true; itd[d] = k + 1; }
            else if (itd[d] == 0) itd[d] = k;
        }
    }
    if (h.dd) dd_store(h, x);
    PR_CUDA(cudaMemcpyAsync(rn.data(), h.rnorm, sizeof(double) * nd, cudaMemcpyDeviceToHost, s));
    PR_CUDA(cudaStreamSynchronize(s));
    BatchSolve out;
    out.iters = k;
    out.outer = k + (x_zero ? 0 : 1);
    for (int d = 0; d < nd; ++d) {
        if (!std::isfinite(rn[d])) fail(PAIR_ERR_NAN, "NaN/Inf in a residual during the AIR solve");
        double rel = bn[d] > 0 ? rn[d] / bn[d] : 0.0;
        out.max_rel = std::max(out.max_rel, rel);
        int kd = std::min(itd[d], k);
        out.cycles += kd;
        if (kd > 0 && r0[d] > 0 && rn[d] > 0) {
            out.rho_sum += std::pow(rn[d] / r0[d], 1.0 / kd);
            out.rho_cnt++;
        }
    }
    out.converged = !any;
    return out;
}

namespace {

__global__ void k_col_count(long long nnz, const int *col, int *cnt) {
    long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < nnz) atomicAdd(&cnt[col[p]], 1);
}

__global__ void k_transpose_scatter(int n, const int *rowptr, const int *col, const double *val, const int *trp,
                                    int *fill, int *tcol, double *tval) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
        int j = col[p];
        int q = trp[j] + atomicAdd(&fill[j], 1);
        tcol[q] = i;
        tval[q] = val[p];
    }
}

// rows of the transpose sorted by column (the scatter order is arbitrary)
__global__ void k_sort_rows(int n, const int *rowptr, int *col, double *val) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int s = rowptr[i], e = rowptr[i + 1];
    for (int a = s + 1; a < e; ++a) {
        int c = col[a];
        double v = val[a];
        int b = a;
        while (b > s && col[b - 1] > c) { col[b] = col[b - 1]; val[b] = val[b - 1]; --b; }
        col[b] = c;
        val[b] = v;
    }
}

// right-hand side of every adjoint direction: the adjoint flux itself
__global__ void k_broadcast(long long N, int nd, const double *v, double *out) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < N * nd) out[t] = v[t % N];
}

// acc += sum_m w_m (W_m^T y_m)  (M c_m with c_m = D_m^{-T} y_m, since M is symmetric);
// NB = DOFs per element (8 for Q1 hexahedra, 4 for P1 tetrahedra)
template <int NB>
__global__ void k_wty_acc(long long E, int nd, const double *W, const double *w, const double *y, double *acc) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= NB * E) return;
    long long e = t / NB;
    int a = (int)(t % NB);
    double s = acc[t];
    for (int m = 0; m < nd; ++m) {
        const double *We = W + ((long long)m * E + e) * NB * NB;
        const double *ye = y + (long long)m * NB * E + NB * e;
        double u = 0.0;
        for (int b = 0; b < NB; ++b) u += We[b * NB + a] * ye[b];
        s += w[m] * u;
    }
    acc[t] = s;
}

// phis_new = g + sigma_s acc / (4 pi)
template <int NB>
__global__ void k_adj_update(long long N, const double *g, const double *sigma_s, const double *acc, double *out) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double inv4pi = 1.0 / (4.0 * 3.14159265358979323846);
    out[i] = g[i] + sigma_s[i / NB] * acc[i] * inv4pi;
}

// per element: dst -= sum_m w_m y^T W psi, dss += sum_m w_m y^T W phi / 4pi, dq += sum_m w_m y^T W 1 / 4pi
template <int NB>
__global__ void k_adj_grad(long long E, int nd, const double *W, const double *w, const double *y, const double *psi,
                           const double *phi, double *dst, double *dss, double *dq) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const double inv4pi = 1.0 / (4.0 * 3.14159265358979323846);
    double gs = dst[e], gss = dss[e], gq = dq[e];
    for (int m = 0; m < nd; ++m) {
        const double *We = W + ((long long)m * E + e) * NB * NB;
        const double *ye = y + (long long)m * NB * E + NB * e;
        const double *pe = psi + (long long)m * NB * E + NB * e;
        const double *fe = phi + NB * e;
        double tp = 0.0, tf = 0.0, t1 = 0.0;
        for (int a = 0; a < NB; ++a) {
            double mp = 0.0, mf = 0.0, m1 = 0.0;
            for (int b = 0; b < NB; ++b) {
                double wab = We[a * NB + b];
                mp += wab * pe[b];
                mf += wab * fe[b];
                m1 += wab;
            }
            tp += ye[a] * mp;
            tf += ye[a] * mf;
            t1 += ye[a] * m1;
        }
        gs -= w[m] * tp;
        gss += w[m] * tf * inv4pi;
        gq += w[m] * t1 * inv4pi;
    }
    dst[e] = gs;
    dss[e] = gss;
    dq[e] = gq;
}

}  // namespace

// Transpose of a CSR matrix (rows sorted by column), on stream s.
void csr_transpose_dev(int n, long long nnz, const int *rowptr, const int *col, const double *val, int *trp,
                       int *tcol, double *tval, cudaStream_t s) {
    int *cnt = dmalloc<int>(n, s);
    PR_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * n, s));
    k_col_count<<<blocks_for(nnz, BS), BS, 0, s>>>(nnz, col, cnt);
    PR_LAUNCH();
    scan_exclusive(cnt, trp, n, s, false);
    PR_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * n, s));
    k_transpose_scatter<<<blocks_for(n, BS), BS, 0, s>>>(n, rowptr, col, val, trp, cnt, tcol, tval);
    PR_LAUNCH();
    k_sort_rows<<<blocks_for(n, BS), BS, 0, s>>>(n, trp, tcol, tval);
    PR_LAUNCH();
    dfree(cnt, s);
}

Hier::~Hier() {
    if (dag) {
        if (stream) dag->release(stream);
        delete dag;
    }
    for (auto &e : ev)
        if (e) cudaEventDestroy(e);
    for (auto &ps : slots) {
        for (auto &e : ps.relax0)
            if (e) cudaEventDestroy(e);
        for (auto &e : ps.res32)
            if (e) cudaEventDestroy(e);
        for (auto &e : ps.lv)
            if (e) cudaEventDestroy(e);
        for (auto &e : ps.lvx)
            if (e) cudaEventDestroy(e);
        for (auto &e : ps.lvt)
            if (e) cudaEventDestroy(e);
    }
    if (stream) {
        for (auto &L : lev) free_level(L, stream);
        void *ptrs[] = {bsr64, bsr32, dsign, partials, rnorm, bnorm, rnorm0, active, d_err, d_n0, d_row00,
                        bsr_dd, b_dd, x_dd, v0, r32, d32, val32, iactive, icount, iany, iticket, ithr, inorm};
        for (void *p : ptrs) dfree(p, stream);
        cudaStreamSynchronize(stream);
        cudaStreamDestroy(stream);
    }
}

// ---- source iteration ---------------------------------------------------------
namespace {

// PAIR_ERR_OOM when the budget (explicit, or the free device memory) cannot hold
// one direction's estimated footprint
void require_budget(size_t per, double avail, bool explicit_budget) {
    if ((double)per <= avail) return;
    char buf[200];
    snprintf(buf, sizeof buf, "%s of %.3f GB is below one direction's estimated footprint of %.3f GB",
             explicit_budget ? "memory budget" : "free device memory", avail * 1e-9, (double)per * 1e-9);
    fail(PAIR_ERR_OOM, buf);
}

// PAIR_ERR_NAN unless every listed device array is finite (checked before any
// kernel consumes the inputs, so NaN never reaches assembly or setup)
void require_finite(std::initializer_list<std::pair<const double *, long long>> arrays, const char *what,
                    cudaStream_t s) {
    int *flag = dmalloc<int>(1, s);
    PR_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), s));
    for (auto &a : arrays) {
        if (!a.first || a.second <= 0) continue;
        unsigned g = std::min<unsigned>(blocks_for(a.second, BS), 152u * 8u);
        k_nonfinite<<<g, BS, 0, s>>>(a.second, a.first, flag);
        PR_LAUNCH();
    }
    int h = 0;
    PR_CUDA(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    dfree(flag, s);
    PR_CUDA(cudaStreamSynchronize(s));
    if (h) fail(PAIR_ERR_NAN, std::string("NaN/Inf in ") + what);
}

__global__ void k_iota_dirs(int nd, long long N, int *row0, int *n0) {
    int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d < nd) { row0[d] = (int)(d * N); n0[d] = (int)N; }
}

size_t bytes_per_dir(const pair_mesh &mesh, int precision, bool gin) {
    bool hex = mesh.kind == PAIR_MESH_HEX;
    size_t nb = hex ? 8 : 4;
    size_t E = hex ? (size_t)mesh.n * mesh.n * mesh.n : (size_t)mesh.ntet, N = nb * E;
    double om[3] = {1, 1, 1};
    size_t nnz0 = hex ? (size_t)hex_nnz(mesh.n, om) : N * 13;
    size_t lvl0 = nnz0 * 12 + (hex ? N * 96 + (precision ? N * 48 : 0) : 0) + E * nb * nb * 8 + (gin ? N * 8 : 0);
    // FP32 inner correction: the FP32 operator copy its residual reads (element-ordered
    // blocks, or CSR values) and its right-hand side and correction
    if (precision) lvl0 += (hex ? N * 48 : nnz0 * 4) + N * 8;
    size_t coarse = nnz0 * 12 * 3 / 2 + nnz0 * 8;   // coarse operators, Z, setup scratch
    // SELL copies (column + value in the cycle precision, ~10% padding) of the coarse
    // levels, of level 0 for the tetrahedral CSR form, and of Z
    coarse += (size_t)((double)(nnz0 * 3 / 2 + (hex ? 0 : nnz0)) * 1.15 + (double)nnz0 / 2) *
              (4 + (precision ? 4 : 8));
    size_t vec = N * (8 * 3 + 4 * 8);
    return lvl0 + coarse + vec;
}

// the exact sweep keeps the level-0 CSR (at most 13 entries per row on either
// mesh), the hex block form or the tet level schedule (< 64 B per element while
// it is built), W, the inflow columns and b, x
size_t sweep_bytes_per_dir(const pair_mesh &mesh, bool gin) {
    bool hex = mesh.kind == PAIR_MESH_HEX;
    size_t nb = hex ? 8 : 4;
    size_t E = hex ? (size_t)mesh.n * mesh.n * mesh.n : (size_t)mesh.ntet, N = nb * E;
    double om[3] = {1, 1, 1};
    size_t nnz0 = hex ? (size_t)hex_nnz(mesh.n, om) : N * 13;
    return nnz0 * 12 + N * 4 + (hex ? N * 96 : E * 64) + E * nb * nb * 8 + (gin ? N * 8 : 0) + N * 16;
}

// a batch of directions m0 .. m0 + nd - 1 (either mesh): its hierarchy or sweep
// schedule, the W and inflow columns of its right-hand sides, and b and x
struct DirBatch {
    int m0 = 0, nd = 0;
    Hier *h = nullptr;
    double *W = nullptr, *Gin = nullptr, *b = nullptr, *xown = nullptr;
};

void free_batch_ops(DirBatch &B) {
    if (!B.h) return;
    cudaStream_t s = B.h->stream;
    dfree(B.W, s); dfree(B.Gin, s);
    B.W = B.Gin = nullptr;
    delete B.h;   // synchronises and destroys its stream
    B.h = nullptr;
}

// device-event kernel timings and algorithmic traffic taken from hierarchies
struct KernelStats {
    double t_res0 = 0, t_relax0 = 0, gb_res0 = 0, gb_relax0 = 0, t_relaxc = 0, gb_relaxc = 0, t_res32 = 0,
           gb_res32 = 0, t_xfer = 0, gb_xfer = 0, t_lvl[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    long long n_res0 = 0, n_relax0 = 0, n_relaxc = 0, n_res32 = 0, n_xfer = 0;
    void take(Hier &h) {   // adds h's counters and clears them
        t_res0 += h.t_res0; t_relax0 += h.t_relax0; gb_res0 += h.gb_res0; gb_relax0 += h.gb_relax0;
        n_res0 += h.n_res0; n_relax0 += h.n_relax0;
        t_relaxc += h.t_relaxc; gb_relaxc += h.gb_relaxc; n_relaxc += h.n_relaxc;
        t_res32 += h.t_res32; gb_res32 += h.gb_res32; n_res32 += h.n_res32;
        t_xfer += h.t_xfer; gb_xfer += h.gb_xfer; n_xfer += h.n_xfer;
        for (int k = 0; k < 8; ++k) { t_lvl[k] += h.t_relaxc_level[k]; h.t_relaxc_level[k] = 0; }
        h.t_res0 = h.t_relax0 = h.gb_res0 = h.gb_relax0 = h.t_relaxc = h.gb_relaxc = h.t_res32 = h.gb_res32 = 0;
        h.t_xfer = h.gb_xfer = 0;
        h.n_res0 = h.n_relax0 = h.n_relaxc = h.n_res32 = h.n_xfer = 0;
    }
    void add(const KernelStats &o) {
        t_res0 += o.t_res0; t_relax0 += o.t_relax0; gb_res0 += o.gb_res0; gb_relax0 += o.gb_relax0;
        t_relaxc += o.t_relaxc; gb_relaxc += o.gb_relaxc; t_res32 += o.t_res32; gb_res32 += o.gb_res32;
        t_xfer += o.t_xfer; gb_xfer += o.gb_xfer;
        for (int k = 0; k < 8; ++k) t_lvl[k] += o.t_lvl[k];
        n_res0 += o.n_res0; n_relax0 += o.n_relax0; n_relaxc += o.n_relaxc; n_res32 += o.n_res32; n_xfer += o.n_xfer;
    }
};

// one batch's share of an SI iteration, merged by the calling thread in batch order
struct BatchOut {
    bool built = false;          // the hierarchy was set up in this iteration
    double setup_ms = 0, solve_ms = 0, tph[4] = {0, 0, 0, 0};
    int levels_max = 0, opc_cnt = 0;
    double opc_sum = 0;
    BatchSolve bs;
    KernelStats ks;
    std::string fail_msg;        // an unconverged solve (with a scalar-flux reduction)
};

// Direction groups solved at the same time, each batch on its own stream from its
// own host thread.  One batch's V-cycle is a chain of dependent launches whose
// coarse levels leave most of the GPU idle (each launch a few microseconds of
// latency for kilobytes of work), and its refinement steps end in host reads; a
// second chain fills those gaps.  Measured on the 32^3 S4 batch (24 directions): one
// batch 256 ms per solve, two concurrent halves 166 ms, three thirds 160 ms.
int auto_concurrency(int M) { return std::min(M, 3); }

void build_batch(DirBatch &B, const pair_mesh &mesh, const double *omega_h, const double *omega_d,
                 const double *sigma_t, const air_params &prm, bool gin, bool adjoint = false,
                 bool sweep_only = false, bool timing = true) {
    const int n = mesh.n;
    const bool hex = mesh.kind == PAIR_MESH_HEX;
    Hier *h = new Hier;
    B.h = h;
    PR_CUDA(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    cudaStream_t s = h->stream;
    int nd = B.nd;
    long long E = hex ? (long long)n * n * n : (long long)mesh.ntet, N = (hex ? 8 : 4) * E;
    h->ndir = nd;
    h->prm = prm;
    h->bsr0 = hex;
    h->hex_n = hex ? n : 0;
    h->n0.assign(nd, (int)N);
    h->d_err = dmalloc<int>(1, s);
    PR_CUDA(cudaMemsetAsync(h->d_err, 0, sizeof(int), s));
    std::vector<int8_t> sg(3 * nd);
    long long nnz = 0;
    for (int d = 0; d < nd; ++d) {
        const double *om = omega_h + 3 * (B.m0 + d);
        for (int k = 0; k < 3; ++k) sg[3 * d + k] = om[k] > 0 ? 1 : (om[k] < 0 ? -1 : 0);
        if (hex) nnz += hex_nnz(n, om);
    }
    h->dsign = dmalloc<int8_t>(3 * nd, s);
    PR_CUDA(cudaMemcpyAsync(h->dsign, sg.data(), 3 * nd, cudaMemcpyHostToDevice, s));
    h->lev.resize(1);
    Level &L = h->lev[0];
    L.n = (int)(N * nd);
    L.rowptr = dmalloc<int>(L.n + 1, s);
    if (!hex)   // entry count depends on the sign of Omega.n on every face
        nnz = tet_assemble(mesh.ntet, nd, omega_d + 3 * B.m0, mesh.verts, mesh.tets, mesh.nbr, sigma_t, L.rowptr,
                           nullptr, nullptr, nullptr, nullptr, h->d_err, s, true);
    PR_REQUIRE(nnz < 0x7fffffffLL, PAIR_ERR_UNSUPPORTED, "direction batch exceeds 2^31 stored entries");
    L.nnz = nnz;
    L.col = dmalloc<int>(nnz, s);
    L.val = dmalloc<double>(nnz, s);
    L.rowdir = dmalloc<int>(L.n, s);
    k_fill_dir<<<blocks_for(L.n, BS), BS, 0, s>>>(L.rowdir, N, nd);
    PR_LAUNCH();
    L.row0.resize(nd);
    L.nrows.assign(nd, (int)N);
    for (int d = 0; d < nd; ++d) L.row0[d] = (int)(d * N);
    L.d_row0 = dmalloc<int>(nd, s);
    h->d_row00 = dmalloc<int>(nd, s);
    h->d_n0 = dmalloc<int>(nd, s);
    k_iota_dirs<<<blocks_for(nd, 64), 64, 0, s>>>(nd, N, L.d_row0, h->d_n0);
    PR_LAUNCH();
    PR_CUDA(cudaMemcpyAsync(h->d_row00, L.d_row0, sizeof(int) * nd, cudaMemcpyDeviceToDevice, s));
    if (hex && !adjoint) {
        h->bsr64 = dmalloc<double>((size_t)nd * E * 96, s);
        if (prm.precision >= 1 && !sweep_only) h->bsr32 = dmalloc<float>((size_t)nd * E * 96, s);
    } else {
        h->bsr0 = false;
    }
    const int nb = hex ? 8 : 4;
    B.W = dmalloc<double>((size_t)nd * E * nb * nb, s);
    if (gin) B.Gin = dmalloc<double>((size_t)nd * N, s);
    if (hex)
        hex_assemble(n, nd, omega_d + 3 * B.m0, sigma_t, L.rowptr, L.col, L.val, h->bsr64, h->bsr32, B.W, B.Gin,
                     h->d_err, s);
    else
        tet_assemble(mesh.ntet, nd, omega_d + 3 * B.m0, mesh.verts, mesh.tets, mesh.nbr, sigma_t, L.rowptr, L.col,
                     L.val, B.W, B.Gin, h->d_err, s, false);
    {   // an element that failed left its rows unwritten: stop before anything reads them
        int aerr = 0;
        PR_CUDA(cudaMemcpyAsync(&aerr, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
        PR_CUDA(cudaStreamSynchronize(s));
        PR_REQUIRE(aerr == 0, PAIR_ERR_SINGULAR,
                   hex ? "assembly: singular element block"
                       : "assembly: zero-volume tetrahedron, singular element block or face-neighbour mismatch");
    }
    if (adjoint) {
        // A_m^T: rows of the transpose of the (block-diagonal) batch operator
        int *trp = dmalloc<int>(L.n + 1, s), *tcol = dmalloc<int>(nnz, s);
        double *tval = dmalloc<double>(nnz, s);
        csr_transpose_dev(L.n, nnz, L.rowptr, L.col, L.val, trp, tcol, tval, s);
        dfree(L.rowptr, s); dfree(L.col, s); dfree(L.val, s);
        L.rowptr = trp; L.col = tcol; L.val = tval;
    }
    if (sweep_only) {   // the exact sweep needs the hex block form or else a level schedule
        if (!(h->bsr0 && h->bsr64)) h->dag = sweep_plan_build(nd, N, nb, L.rowptr, L.col, h->d_err, s);
        PR_CUDA(cudaStreamSynchronize(s));
        return;
    }
    build_hierarchy(*h);
    alloc_cycle_vectors(*h);
    dd_enable(*h);
    inner_enable(*h);
    split0_enable(*h);
    level0_bytes(*h);
    if (timing) prof_enable(*h);
}

}  // namespace

void si_run(const pair_mesh &mesh, const pair_quad &quad, const double *sigma_t, const double *sigma_s,
            const double *q, const air_params &prm, const si_params &sp, double *phi, double *psi,
            cudaStream_t user, si_info *info) {
    int n = mesh.n, M = quad.M;
    const bool hex = mesh.kind == PAIR_MESH_HEX;
    const int nbk0 = hex ? 8 : 4;
    long long E = hex ? (long long)n * n * n : (long long)mesh.ntet, N = nbk0 * E;
    PR_CUDA(cudaStreamSynchronize(user));
    bool gin = sp.g_inflow != 0.0;
    const bool sweep = sp.solver == 1;
    // direction batches admitted by memory
    size_t per = sweep ? sweep_bytes_per_dir(mesh, gin) : bytes_per_dir(mesh, prm.precision, gin);
    const size_t freeb = available_device_bytes();
    double budget = sp.mem_budget_gb > 0 ? sp.mem_budget_gb * 1e9 : 0.6 * (double)freeb;
    require_budget(per, sp.mem_budget_gb > 0 ? budget : (double)freeb, sp.mem_budget_gb > 0);
    int B = sp.batch > 0 ? std::min(sp.batch, M) : M;
    B = std::min<long long>(B, std::max<long long>(1, (long long)(budget / (double)per)));
    // 32-bit entry indices: a hierarchy's levels hold up to ~64 entries per level-0
    // row in total, the sweep's level-0 CSR at most 13
    B = (int)std::min<long long>(B, std::max<long long>(1, (0x7fffffffLL / (sweep ? 16 : 64)) / N));
    int nb = (M + B - 1) / B;
    bool resident = (double)per * M <= budget;
    // concurrent direction groups (resident hierarchies only: a rebuilt batch is
    // sized to the whole budget); the directions are split so each group has a batch
    int K = 1;
    if (resident && !sweep) {
        K = std::max(1, std::min(sp.concurrent > 0 ? sp.concurrent : auto_concurrency(M), M));
        if (nb < K) {
            B = (M + K - 1) / K;
            nb = (M + B - 1) / B;
        }
        K = std::min(K, nb);
    }
    int dev = 0;
    PR_CUDA(cudaGetDevice(&dev));
    // per-call device state on a private stream
    cudaStream_t s;
    PR_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    struct Cleanup {
        cudaStream_t s;
        std::vector<DirBatch> *bs;
        std::vector<void *> bufs;
        ~Cleanup() {
            for (auto &b : *bs) {
                if (b.h) { dfree(b.b, b.h->stream); dfree(b.xown, b.h->stream); }
                free_batch_ops(b);
            }
            for (void *p : bufs) cudaFreeAsync(p, s);
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
    };
    std::vector<DirBatch> batches(nb);
    Cleanup cl{s, &batches, {}};
    require_finite({{sigma_t, E}, {sigma_s, E}, {q, E}, {phi, N}, {sp.q_ang, sp.q_ang ? N * M : 0}},
                   "sigma_t, sigma_s, q, the initial phi or q_ang", s);
    double *omega_d = dmalloc<double>(3 * M, s);
    cl.bufs.push_back(omega_d);
    PR_CUDA(cudaMemcpyAsync(omega_d, quad.omega, sizeof(double) * 3 * M, cudaMemcpyHostToDevice, s));
    double *w_d = dmalloc<double>(M, s);
    cl.bufs.push_back(w_d);
    PR_CUDA(cudaMemcpyAsync(w_d, quad.w, sizeof(double) * M, cudaMemcpyHostToDevice, s));
    // the new flux, and one status slot for the reduction of a direction subset
    double *phinew = dmalloc<double>(N + 1, s);
    cl.bufs.push_back(phinew);
    double *src = dmalloc<double>(N, s);   // isotropic source of the current iteration
    cl.bufs.push_back(src);
    int nbk = (int)blocks_for(N, BS);
    double *part = dmalloc<double>(2 * (size_t)nbk, s);
    cl.bufs.push_back(part);
    double *dres = dmalloc<double>(2, s);
    cl.bufs.push_back(dres);
    // partial fluxes of the concurrent groups, summed in group order
    double *partial = nullptr;
    if (K > 1) {
        partial = dmalloc<double>((size_t)K * N, s);
        cl.bufs.push_back(partial);
    }
    PR_CUDA(cudaStreamSynchronize(s));
    for (int b = 0; b < nb; ++b) { batches[b].m0 = b * B; batches[b].nd = std::min(B, M - b * B); }

    cudaEvent_t e0, e1, ev_src;
    PR_CUDA(cudaEventCreate(&e0));
    PR_CUDA(cudaEventCreate(&e1));
    PR_CUDA(cudaEventCreateWithFlags(&ev_src, cudaEventDisableTiming));
    struct Events {
        cudaEvent_t e[3];
        ~Events() {
            for (auto x : e)
                if (x) cudaEventDestroy(x);
        }
    } evs{{e0, e1, ev_src}};
    double t_setup = 0, t_solve = 0;
    int vcycles = 0, levels_max = 0;
    double max_inner = 0, opc_sum = 0, change = 0;
    int opc_cnt = 0, it = 0;
    double tph[4] = {0, 0, 0, 0};
    long long outer_res = 0;
    KernelStats ks;
    bool converged = false, timed_it = false;
    int timed_iters = 0;
    // One batch's share of an iteration: setup on first use, right-hand sides from
    // the iteration's source, the direction solves, and sum_m w_m psi_m into acc
    // (written when 'overwrite', else added).  Runs on the calling thread or on a
    // group's thread; everything it reports goes to 'o'.
    auto run_batch = [&](int bi, double *acc, bool overwrite, BatchOut &o) {
        DirBatch &Bt = batches[bi];
        if (!Bt.h) {
            auto t0 = std::chrono::steady_clock::now();
            build_batch(Bt, mesh, quad.omega, omega_d, sigma_t, prm, gin, false, sweep, sp.timing != 0);
            PR_CUDA(cudaStreamSynchronize(Bt.h->stream));
            o.setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            o.built = true;
            for (int k = 0; k < 4; ++k) o.tph[k] = Bt.h->t_phase[k];
            cudaStream_t hs = Bt.h->stream;
            Bt.b = dmalloc<double>((size_t)Bt.nd * N, hs);
            if (!psi) Bt.xown = dmalloc<double>((size_t)Bt.nd * N, hs);
            Hier &h = *Bt.h;
            for (int d = 0; d < Bt.nd && !sweep; ++d) {
                int nl = 0;
                long long tot = 0;
                for (auto &L : h.lev)
                    if (L.nrows.size() && L.nrows[d] > 0) { ++nl; tot += L.nnzdir[d]; }
                o.levels_max = std::max(o.levels_max, nl);
                o.opc_sum += (double)tot / (double)h.lev[0].nnzdir[d];
                ++o.opc_cnt;
            }
        }
        Hier &h = *Bt.h;
        cudaStream_t hs = h.stream;
        h.timed = h.prof && timed_it;
        double *x = psi ? psi + (size_t)Bt.m0 * N : Bt.xown;
        const double *qa = sp.q_ang ? sp.q_ang + (size_t)Bt.m0 * N : nullptr;
        cudaEvent_t a, z;
        PR_CUDA(cudaEventCreate(&a));
        Events own{{a, nullptr, nullptr}};
        PR_CUDA(cudaEventCreate(&z));
        own.e[1] = z;
        PR_CUDA(cudaEventRecord(a, hs));
        PR_CUDA(cudaStreamWaitEvent(hs, ev_src, 0));
        if (hex)
            k_rhs<8><<<blocks_for((long long)Bt.nd * N, BS), BS, 0, hs>>>(E, Bt.nd, Bt.W, Bt.Gin, sp.g_inflow, src,
                                                                       qa, Bt.b);
        else
            k_rhs<4><<<blocks_for((long long)Bt.nd * N, BS), BS, 0, hs>>>(E, Bt.nd, Bt.W, Bt.Gin, sp.g_inflow, src,
                                                                       qa, Bt.b);
        PR_LAUNCH();
        BatchSolve bs;
        if (sweep) {
            sweep_solve(h, Bt.b, x, sp.use_graphs != 0);
            bs.converged = true;
        } else {
            PR_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * Bt.nd * N, hs));
            if (sp.inner_cycles > 0) {   // fixed approximate inverse: l cycles from zero
                bs = solve_batch(h, Bt.b, x, 0.0, sp.inner_cycles, sp.use_graphs != 0, true);
                bs.converged = true;
            } else {
                bs = solve_batch(h, Bt.b, x, sp.inner_tol, sp.inner_maxit, sp.use_graphs != 0, true);
            }
        }
        if (!bs.converged) {
            char buf[160];
            snprintf(buf, sizeof buf, "AIR solve reached %d cycles with relative residual %.3e > %.3e", bs.iters,
                     bs.max_rel, sp.inner_tol);
            // with a reduction the other processes wait for this one: report after it
            if (!sp.phi_reduce) fail(PAIR_ERR_NOT_CONVERGED, buf);
            o.fail_msg = buf;
        }
        o.bs = bs;
        k_phi_acc<<<blocks_for(N, BS), BS, 0, hs>>>(N, Bt.nd, w_d + Bt.m0, x, acc, overwrite ? 1 : 0);
        PR_LAUNCH();
        PR_CUDA(cudaEventRecord(z, hs));
        PR_CUDA(cudaEventSynchronize(z));
        float ms = 0;
        PR_CUDA(cudaEventElapsedTime(&ms, a, z));
        o.solve_ms = ms;
        o.ks.take(h);
        if (!resident) {
            dfree(Bt.b, hs); dfree(Bt.xown, hs);
            Bt.b = Bt.xown = nullptr;
            free_batch_ops(Bt);
        }
    };
    std::string local_fail;   // with a reduction: the first unconverged solve of this iteration
    for (it = 0; it < sp.max_iters; ++it) {
        // SI iterations k, 2k, ... (counting from 1) record the kernel timings, with the
        // groups one after another so that no other group's kernels share their events
        timed_it = sp.timing > 0 && (it + 1) % sp.timing == 0;
        if (timed_it) ++timed_iters;
        PR_CUDA(cudaMemsetAsync(phinew, 0, sizeof(double) * (N + 1), s));
        PR_CUDA(cudaEventRecord(e0, s));
        // the source of this iteration, once for every batch
        if (hex) k_src<8><<<blocks_for(N, BS), BS, 0, s>>>(N, sigma_s, q, phi, src);
        else k_src<4><<<blocks_for(N, BS), BS, 0, s>>>(N, sigma_s, q, phi, src);
        PR_LAUNCH();
        PR_CUDA(cudaEventRecord(ev_src, s));
        PR_CUDA(cudaStreamSynchronize(s));
        local_fail.clear();
        std::vector<BatchOut> outs(nb);
        if (K == 1) {
            for (int bi = 0; bi < nb; ++bi) run_batch(bi, phinew, false, outs[bi]);
        } else if (timed_it) {
            for (int k = 0; k < K; ++k)
                for (int bi = k; bi < nb; bi += K) run_batch(bi, partial + (size_t)k * N, bi == k, outs[bi]);
            k_phi_sum<<<blocks_for(N, BS), BS, 0, s>>>(N, K, partial, phinew);
            PR_LAUNCH();
        } else {
            // group k takes batches k, k + K, ... in order, summing into its partial
            std::vector<std::exception_ptr> errs(K);
            std::vector<std::thread> th;
            for (int k = 0; k < K; ++k)
                th.emplace_back([&, k] {
                    try {
                        PR_CUDA(cudaSetDevice(dev));
                        for (int bi = k; bi < nb; bi += K) run_batch(bi, partial + (size_t)k * N, bi == k, outs[bi]);
                    } catch (...) {
                        errs[k] = std::current_exception();
                    }
                });
            for (auto &t : th) t.join();
            for (auto &e : errs)
                if (e) std::rethrow_exception(e);
            // every group's stream was synchronised when its thread finished
            k_phi_sum<<<blocks_for(N, BS), BS, 0, s>>>(N, K, partial, phinew);
            PR_LAUNCH();
        }
        // merge in batch order
        double setup_max = 0, setup_sum = 0, solve_sum = 0;
        int longest = -1;
        for (int bi = 0; bi < nb; ++bi) {
            BatchOut &o = outs[bi];
            if (o.built) {
                setup_sum += o.setup_ms;
                if (longest < 0 || o.setup_ms > setup_max) { setup_max = o.setup_ms; longest = bi; }
                levels_max = std::max(levels_max, o.levels_max);
                opc_sum += o.opc_sum;
                opc_cnt += o.opc_cnt;
            }
            solve_sum += o.solve_ms;
            vcycles += (int)o.bs.cycles;
            outer_res += o.bs.outer;
            max_inner = std::max(max_inner, o.bs.max_rel);
            ks.add(o.ks);
            if (local_fail.empty() && !o.fail_msg.empty()) local_fail = o.fail_msg;
        }
        if (K == 1) {   // batches one after the other: their times add
            t_setup += setup_sum;
            t_solve += solve_sum;
            for (int bi = 0; bi < nb; ++bi)
                for (int k = 0; k < 4; ++k) tph[k] += outs[bi].tph[k];
        } else {        // concurrent groups: the iteration's wall time, setup = the longest batch setup
            PR_CUDA(cudaEventRecord(e1, s));
            PR_CUDA(cudaEventSynchronize(e1));
            float wall = 0;
            PR_CUDA(cudaEventElapsedTime(&wall, e0, e1));
            t_setup += setup_max;
            t_solve += std::max(0.0, (double)wall - setup_max);
            if (longest >= 0)
                for (int k = 0; k < 4; ++k) tph[k] += outs[longest].tph[k];
        }
        if (sp.phi_reduce) {   // angular decomposition: sum the partial fluxes and statuses
            const double st = local_fail.empty() ? 0.0 : 1.0;
            PR_CUDA(cudaMemcpyAsync(phinew + N, &st, sizeof(double), cudaMemcpyHostToDevice, s));
            PR_CUDA(cudaStreamSynchronize(s));
            const int rc = sp.phi_reduce(phinew, N + 1, sp.reduce_ctx);
            PR_REQUIRE(rc == 0, PAIR_ERR_COMM, "scalar-flux reduction returned " + std::to_string(rc));
            double tot = 0;
            PR_CUDA(cudaMemcpyAsync(&tot, phinew + N, sizeof(double), cudaMemcpyDeviceToHost, s));
            PR_CUDA(cudaStreamSynchronize(s));
            if (tot > 0)
                fail(PAIR_ERR_NOT_CONVERGED, local_fail.empty() ? "a direction solve of another process missed "
                                                                  "inner_tol"
                                                                : local_fail);
        }
        k_diff_partials<<<nbk, BS, 0, s>>>(N, phinew, phi, part);
        PR_LAUNCH();
        k_diff_final<<<1, DIFF_BS, 0, s>>>(nbk, part, dres);
        PR_LAUNCH();
        double hr[2];
        PR_CUDA(cudaMemcpyAsync(hr, dres, sizeof hr, cudaMemcpyDeviceToHost, s));
        PR_CUDA(cudaMemcpyAsync(phi, phinew, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
        PR_CUDA(cudaStreamSynchronize(s));
        change = hr[1] > 0 ? hr[0] / hr[1] : 0.0;
        if (!std::isfinite(change)) fail(PAIR_ERR_NAN, "NaN/Inf in the scalar flux");
        if (change <= sp.tol) { converged = true; ++it; break; }
    }
    if (info) {
        info->si_iters = std::min(it, sp.max_iters);
        info->si_change = change;
        info->vcycles = vcycles;
        info->max_inner_resid = max_inner;
        info->batches = nb;
        info->rebuilt = resident ? 0 : 1;
        info->t_setup_ms = t_setup;
        info->t_solve_ms = t_solve;
        info->levels_max = levels_max;
        info->op_complexity = opc_cnt ? opc_sum / opc_cnt : 0;
        info->t_res0_ms = ks.t_res0;
        info->n_res0 = (int)ks.n_res0;
        info->gb_res0 = ks.gb_res0;
        info->t_relax0_ms = ks.t_relax0;
        info->n_relax0 = (int)ks.n_relax0;
        info->gb_relax0 = ks.gb_relax0;
        info->t_relaxc_ms = ks.t_relaxc;
        info->n_relaxc = (int)ks.n_relaxc;
        info->gb_relaxc = ks.gb_relaxc;
        info->t_res32_ms = ks.t_res32;
        info->n_res32 = (int)ks.n_res32;
        info->gb_res32 = ks.gb_res32;
        info->outer_residuals = (int)outer_res;
        for (int k = 0; k < 8; ++k) info->t_relaxc_level_ms[k] = ks.t_lvl[k];
        info->timed_iters = timed_iters;
        info->t_xfer_ms = ks.t_xfer;
        info->n_xfer = (int)ks.n_xfer;
        info->gb_xfer = ks.gb_xfer;
        for (int k = 0; k < 3; ++k) info->t_setup_phase_ms[k] = tph[k];
        info->t_setup_phase_ms[3] = t_setup - (tph[0] + tph[1] + tph[2]);
    }
    if (!converged && sp.max_iters > 1 && !sp.fixed_iters) {
        char buf[128];
        snprintf(buf, sizeof buf, "source iteration: %d iterations, change %.3e > %.3e", sp.max_iters, change, sp.tol);
        fail(PAIR_ERR_NOT_CONVERGED, buf);
    }
}

void si_adjoint_run(const pair_mesh &mesh, const pair_quad &quad, const double *sigma_t, const double *sigma_s,
                    const double *psi, const double *g, const air_params &prm, const si_params &sp, double *dst,
                    double *dss, double *dq, double *phis_out, cudaStream_t user, si_info *info) {
    const bool hex = mesh.kind == PAIR_MESH_HEX;
    int M = quad.M;
    long long E = hex ? (long long)mesh.n * mesh.n * mesh.n : (long long)mesh.ntet, N = (hex ? 8 : 4) * E;
    const bool sweep = sp.solver == 1;   // exact sweeps of the transposed operators instead of AIR
    PR_CUDA(cudaStreamSynchronize(user));
    size_t per = (sweep ? sweep_bytes_per_dir(mesh, false) : bytes_per_dir(mesh, prm.precision, false)) + (size_t)N * 16;
    const size_t freeb = available_device_bytes();
    double budget = sp.mem_budget_gb > 0 ? sp.mem_budget_gb * 1e9 : 0.6 * (double)freeb;
    int B = sp.batch > 0 ? std::min(sp.batch, M) : M;
    B = std::min<long long>(B, std::max<long long>(1, (long long)(budget / (double)per)));
    B = (int)std::min<long long>(B, std::max<long long>(1, (0x7fffffffLL / 64) / N));
    int nb = (M + B - 1) / B;
    bool resident = (double)per * M <= budget;
    PR_REQUIRE(resident, PAIR_ERR_OOM, "si_adjoint: all direction hierarchies must fit the memory budget");
    int K = 1;   // concurrent direction groups, as in si_run
    if (!sweep) {
        K = std::max(1, std::min(sp.concurrent > 0 ? sp.concurrent : auto_concurrency(M), M));
        if (nb < K) {
            B = (M + K - 1) / K;
            nb = (M + B - 1) / B;
        }
        K = std::min(K, nb);
    }
    int dev = 0;
    PR_CUDA(cudaGetDevice(&dev));
    cudaStream_t s;
    PR_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    std::vector<DirBatch> batches(nb);
    struct Cleanup {
        cudaStream_t s;
        std::vector<DirBatch> *bs;
        std::vector<void *> bufs;
        ~Cleanup() {
            for (auto &b : *bs) {
                if (b.h) { dfree(b.b, b.h->stream); dfree(b.xown, b.h->stream); }
                free_batch_ops(b);
            }
            for (void *p : bufs) cudaFreeAsync(p, s);
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
    } cl{s, &batches, {}};
    require_finite({{sigma_t, E}, {sigma_s, E}, {psi, N * M}, {g, N}}, "sigma_t, sigma_s, psi or g", s);
    auto buf = [&](size_t cnt) { double *p = dmalloc<double>(cnt, s); cl.bufs.push_back(p); return p; };
    double *omega_d = buf(3 * M), *w_d = buf(M), *phi = buf(N), *phis = buf(N), *pnew = buf(N), *acc = buf(N);
    int nbk = (int)blocks_for(N, BS);
    double *part = buf(2 * (size_t)nbk), *dres = buf(2);
    double *partial = K > 1 ? buf((size_t)K * N) : nullptr;   // the groups' sums
    PR_CUDA(cudaMemcpyAsync(omega_d, quad.omega, sizeof(double) * 3 * M, cudaMemcpyHostToDevice, s));
    PR_CUDA(cudaMemcpyAsync(w_d, quad.w, sizeof(double) * M, cudaMemcpyHostToDevice, s));
    PR_CUDA(cudaMemsetAsync(phi, 0, sizeof(double) * N, s));
    PR_CUDA(cudaMemsetAsync(phis, 0, sizeof(double) * N, s));
    // forward scalar flux from the given angular fluxes
    k_phi_acc<<<blocks_for(N, BS), BS, 0, s>>>(N, M, w_d, psi, phi, 0);
    PR_LAUNCH();
    PR_CUDA(cudaStreamSynchronize(s));
    cudaEvent_t e0, e1;
    PR_CUDA(cudaEventCreate(&e0));
    PR_CUDA(cudaEventCreate(&e1));
    double t_setup = 0, t_solve = 0, change = 0, max_inner = 0;
    int vcycles = 0, it = 0;
    bool converged = false;
    // K groups run their batches k, k + K, ... on their own threads (K = 1: this thread)
    auto in_groups = [&](auto &&work) {
        if (K == 1) {
            for (int b = 0; b < nb; ++b) work(b, 0);
            return;
        }
        std::vector<std::exception_ptr> errs(K);
        std::vector<std::thread> th;
        for (int k = 0; k < K; ++k)
            th.emplace_back([&, k] {
                try {
                    PR_CUDA(cudaSetDevice(dev));
                    for (int b = k; b < nb; b += K) work(b, k);
                } catch (...) {
                    errs[k] = std::current_exception();
                }
            });
        for (auto &t : th) t.join();
        for (auto &e : errs)
            if (e) std::rethrow_exception(e);
    };
    for (int b = 0; b < nb; ++b) { batches[b].m0 = b * B; batches[b].nd = std::min(B, M - b * B); }
    {
        auto t0 = std::chrono::steady_clock::now();
        in_groups([&](int b, int) {
            DirBatch &Bt = batches[b];
            build_batch(Bt, mesh, quad.omega, omega_d, sigma_t, prm, false, true, sweep, false);
            cudaStream_t hs = Bt.h->stream;
            Bt.b = dmalloc<double>((size_t)Bt.nd * N, hs);
            Bt.xown = dmalloc<double>((size_t)Bt.nd * N, hs);
            PR_CUDA(cudaStreamSynchronize(hs));
        });
        t_setup = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    std::vector<BatchSolve> bsv(nb);
    for (it = 0; it < sp.max_iters; ++it) {
        PR_CUDA(cudaMemsetAsync(acc, 0, sizeof(double) * N, s));
        if (K > 1) PR_CUDA(cudaMemsetAsync(partial, 0, sizeof(double) * K * N, s));
        PR_CUDA(cudaEventRecord(e0, s));
        PR_CUDA(cudaStreamSynchronize(s));
        // each batch adds sum_m w_m W_m^T lambda_m into its group's sum (K = 1: acc)
        in_groups([&](int b, int k) {
            DirBatch &Bt = batches[b];
            Hier &h = *Bt.h;
            cudaStream_t hs = h.stream;
            double *dst_acc = K > 1 ? partial + (size_t)k * N : acc;
            k_broadcast<<<blocks_for((long long)Bt.nd * N, BS), BS, 0, hs>>>(N, Bt.nd, phis, Bt.b);
            PR_LAUNCH();
            BatchSolve bs;
            if (sweep) {
                sweep_solve(h, Bt.b, Bt.xown, sp.use_graphs != 0);
            } else {
                PR_CUDA(cudaMemsetAsync(Bt.xown, 0, sizeof(double) * Bt.nd * N, hs));
                bs = solve_batch(h, Bt.b, Bt.xown, sp.inner_tol, sp.inner_maxit, sp.use_graphs != 0, true);
            }
            if (!bs.converged && it > 0) {   // the first right-hand side is zero
                char buf2[160];
                snprintf(buf2, sizeof buf2, "adjoint AIR solve reached %d cycles with relative residual %.3e",
                         bs.iters, bs.max_rel);
                fail(PAIR_ERR_NOT_CONVERGED, buf2);
            }
            bsv[b] = bs;
            if (hex)
                k_wty_acc<8><<<blocks_for(N, BS), BS, 0, hs>>>(E, Bt.nd, Bt.W, w_d + Bt.m0, Bt.xown, dst_acc);
            else
                k_wty_acc<4><<<blocks_for(N, BS), BS, 0, hs>>>(E, Bt.nd, Bt.W, w_d + Bt.m0, Bt.xown, dst_acc);
            PR_LAUNCH();
            PR_CUDA(cudaStreamSynchronize(hs));
        });
        if (K > 1) {
            k_phi_sum<<<blocks_for(N, BS), BS, 0, s>>>(N, K, partial, acc);
            PR_LAUNCH();
        }
        for (int b = 0; b < nb; ++b) {
            vcycles += (int)bsv[b].cycles;
            max_inner = std::max(max_inner, bsv[b].max_rel);
        }
        PR_CUDA(cudaEventRecord(e1, s));
        PR_CUDA(cudaEventSynchronize(e1));
        float ms = 0;
        PR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        t_solve += ms;
        if (hex)
            k_adj_update<8><<<blocks_for(N, BS), BS, 0, s>>>(N, g, sigma_s, acc, pnew);
        else
            k_adj_update<4><<<blocks_for(N, BS), BS, 0, s>>>(N, g, sigma_s, acc, pnew);
        PR_LAUNCH();
        k_diff_partials<<<nbk, BS, 0, s>>>(N, pnew, phis, part);
        PR_LAUNCH();
        k_diff_final<<<1, DIFF_BS, 0, s>>>(nbk, part, dres);
        PR_LAUNCH();
        double hr[2];
        PR_CUDA(cudaMemcpyAsync(hr, dres, sizeof hr, cudaMemcpyDeviceToHost, s));
        PR_CUDA(cudaMemcpyAsync(phis, pnew, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
        PR_CUDA(cudaStreamSynchronize(s));
        change = hr[1] > 0 ? hr[0] / hr[1] : 0.0;
        if (!std::isfinite(change)) fail(PAIR_ERR_NAN, "NaN/Inf in the adjoint flux");
        if (change <= sp.tol) { converged = true; ++it; break; }
    }
    // gradients from the last adjoint solutions
    PR_CUDA(cudaMemsetAsync(dst, 0, sizeof(double) * E, s));
    PR_CUDA(cudaMemsetAsync(dss, 0, sizeof(double) * E, s));
    PR_CUDA(cudaMemsetAsync(dq, 0, sizeof(double) * E, s));
    PR_CUDA(cudaStreamSynchronize(s));
    for (int b = 0; b < nb; ++b) {
        DirBatch &Bt = batches[b];
        if (hex)
            k_adj_grad<8><<<blocks_for(E, 128), 128, 0, s>>>(E, Bt.nd, Bt.W, w_d + Bt.m0, Bt.xown,
                                                             psi + (size_t)Bt.m0 * N, phi, dst, dss, dq);
        else
            k_adj_grad<4><<<blocks_for(E, 128), 128, 0, s>>>(E, Bt.nd, Bt.W, w_d + Bt.m0, Bt.xown,
                                                             psi + (size_t)Bt.m0 * N, phi, dst, dss, dq);
        PR_LAUNCH();
    }
    if (phis_out) PR_CUDA(cudaMemcpyAsync(phis_out, phis, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    PR_CUDA(cudaStreamSynchronize(s));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (info) {
        memset(info, 0, sizeof(*info));
        info->si_iters = std::min(it, sp.max_iters);
        info->si_change = change;
        info->vcycles = vcycles;
        info->max_inner_resid = max_inner;
        info->batches = nb;
        info->t_setup_ms = t_setup;
        info->t_solve_ms = t_solve;
    }
    if (!converged && sp.max_iters > 1) {
        char buf2[128];
        snprintf(buf2, sizeof buf2, "adjoint source iteration: %d iterations, change %.3e > %.3e", sp.max_iters,
                 change, sp.tol);
        fail(PAIR_ERR_NOT_CONVERGED, buf2);
    }
}

}  // namespace pr
