// Exact solve of the block-scaled upwind DG system of every direction of a batch by
// a GPU sweep (Sec. 1.1: the transport sweep; Sec. 6 compares pAIR with sweeps).
//
// After block-inverse scaling (Sec. 1.3) the diagonal blocks are identities, so for
// an element e the unknowns follow from its upwind neighbours alone:
//     x_e = b_e - sum_{upwind faces f} A_ef x_f.
// On the structured hex mesh the elements with the same upwind-ordered index sum
// ix' + iy' + iz' (ix' = ix where Omega_x > 0, n - 1 - ix where Omega_x < 0; any
// order on an axis with Omega_x = 0, which carries no coupling) depend only on
// earlier sums, so the solve is 3n - 2 dependent wavefronts.  One launch per
// wavefront covers every direction of the batch (8 threads per element, one per
// node); the launches are captured once into a CUDA graph per batch and use
// programmatic dependent launch, so a wavefront starts as the previous one drains.
// Batches without the structured block form (tetrahedra, transposed operators)
// take the level schedule of sweep_dag.cu through the same entry point.
#include "common.cuh"

namespace pr {

namespace {

constexpr int SW_BS = 256;

__device__ __forceinline__ int sw_face_node(int d, int o, int t) {
    return d == 0 ? (o | (t << 1)) : d == 1 ? ((t & 1) | (o << 1) | ((t >> 1) << 2)) : (t | (o << 2));
}

__global__ void __launch_bounds__(SW_BS) k_sweep_wave(int n, int N, int wave, const int8_t *dsign,
                                                      const double *bsr64, const double *b, double *x) {
    pdl_begin();
    const int m = blockIdx.y;
    const long long t = (long long)blockIdx.x * SW_BS + threadIdx.x;
    const long long pair = t >> 3;
    const int a = (int)(t & 7);
    if (pair >= (long long)n * n) return;
    const int ixp = (int)(pair % n), iyp = (int)(pair / n);
    const int izp = wave - ixp - iyp;
    if (izp < 0 || izp >= n) return;
    const int sg[3] = {dsign[3 * m], dsign[3 * m + 1], dsign[3 * m + 2]};
    const int idx[3] = {sg[0] >= 0 ? ixp : n - 1 - ixp, sg[1] >= 0 ? iyp : n - 1 - iyp,
                        sg[2] >= 0 ? izp : n - 1 - izp};
    const int stride[3] = {1, n, n * n};
    const long long E = (long long)N / 8;
    const int e = idx[0] + n * (idx[1] + n * idx[2]);
    const double *base = bsr64 + (((long long)m * E + e) * 3) * 32 + a * 4;
    const double *xm = x + (long long)m * N;
    double acc = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (sg[d] == 0) continue;
        const bool has = sg[d] > 0 ? idx[d] > 0 : idx[d] < n - 1;
        if (!has) continue;
        const int ep = sg[d] > 0 ? e - stride[d] : e + stride[d];
        const int o = sg[d] > 0 ? 1 : 0;
        const double *w = base + d * 32;
        const double *xb = xm + 8LL * ep;
#pragma unroll
        for (int k = 0; k < 4; ++k) acc += w[k] * xb[sw_face_node(d, o, k)];
    }
    const long long gi = (long long)m * N + 8LL * e + a;
    x[gi] = b[gi] - acc;
}

void launch_waves(Hier &h, const double *b, double *x) {
    const int n = h.hex_n, N = h.n0[0];
    const dim3 grid(blocks_for(8LL * n * n, SW_BS), h.ndir);
    for (int w = 0; w <= 3 * (n - 1); ++w) {
        launch_pdl(k_sweep_wave, grid, dim3(SW_BS), h.stream, n, N, w, (const int8_t *)h.dsign,
                   (const double *)h.bsr64, b, x);
        PR_LAUNCH();
    }
}

void launch_sweep(Hier &h, const double *b, double *x) {
    if (h.bsr0 && h.bsr64) {
        launch_waves(h, b, x);
    } else {
        const Level &L = h.lev[0];
        sweep_plan_launch(*h.dag, L.rowptr, L.col, L.val, b, x, h.d_err, h.stream);
    }
}

}  // namespace

// Structured hex batches (block form present) take the wavefront sweep, every
// other batch the level schedule built with it (sweep_dag.cu).
void sweep_solve(Hier &h, const double *b, double *x, bool use_graph) {
    PR_REQUIRE((h.bsr0 && h.bsr64) || h.dag, PAIR_ERR_UNSUPPORTED, "GPU sweep: no block form or level schedule");
    if (!use_graph) {
        launch_sweep(h, b, x);
        return;
    }
    CycleGraphs &G = h.gr[0];   // a sweep records no timing events
    if (!G.graph || G.graph_b != b || G.graph_x != x) {
        if (G.graph) { cudaGraphExecDestroy(G.graph); G.graph = nullptr; }
        cudaGraph_t g;
        const long long before = g_thread_launches;
        PR_CUDA(cudaStreamBeginCapture(h.stream, cudaStreamCaptureModeThreadLocal));
        try {
            launch_sweep(h, b, x);
        } catch (...) {
            cudaGraph_t dummy = nullptr;
            cudaStreamEndCapture(h.stream, &dummy);
            if (dummy) cudaGraphDestroy(dummy);
            g_launches -= g_thread_launches - before;
            throw;
        }
        PR_CUDA(cudaStreamEndCapture(h.stream, &g));
        G.graph_kernels = g_thread_launches - before;
        g_launches -= G.graph_kernels;   // counted per replay instead
        PR_CUDA(cudaGraphInstantiate(&G.graph, g, 0));
        cudaGraphDestroy(g);
        G.graph_b = b;
        G.graph_x = x;
        G.graph_tol = -2.0;
    }
    PR_CUDA(cudaGraphLaunch(G.graph, h.stream));
    g_launches += G.graph_kernels;
}

}  // namespace pr
