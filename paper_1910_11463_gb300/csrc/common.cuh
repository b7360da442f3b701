// Internal declarations of libpair (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/pair.h"

namespace pr {

struct Error {
    pair_status st;
    std::string msg;
};

[[noreturn]] void fail(pair_status st, const std::string &msg);
void set_last_error(const std::string &msg);   // the message pair_last_error() returns
void cuda_check(cudaError_t e, const char *what, const char *file, int line);

#define PR_CUDA(call) ::pr::cuda_check((call), #call, __FILE__, __LINE__)
// Every kernel launch of the library is followed by PR_LAUNCH(), which also
// counts it: in the process-wide count (launches recorded while capturing a graph
// are counted per replay instead) and in the calling thread's own count, which a
// capture uses to size its graph while other threads launch work.
extern std::atomic<long long> g_launches;
extern thread_local long long g_thread_launches;
#define PR_LAUNCH() \
    (++::pr::g_launches, ++::pr::g_thread_launches, \
     ::pr::cuda_check(cudaGetLastError(), "kernel launch", __FILE__, __LINE__))
#define PR_REQUIRE(cond, st, msg) \
    do {                          \
        if (!(cond)) ::pr::fail((st), (msg)); \
    } while (0)

// Device error word bits (set by kernels, read by the host after a phase).
enum : int {
    DERR_HASH_OVERFLOW = 1,
    DERR_PATTERN_TOO_LARGE = 2,
    DERR_BOUNDS = 4,
    DERR_SWEEP = 16,   // sweep plan limits (faces per element, cyclic components) or a singular component
};

// The library's stream-ordered memory pool on the current device: created on first
// use with no release threshold, so memory a call frees stays mapped for the next
// call's allocations (a complete solve allocates and frees gigabytes of hierarchy
// and setup scratch; without this every call would map them afresh).  The pool's
// memory returns to the system when the process exits.
cudaMemPool_t device_pool();
size_t available_device_bytes();   // free device memory plus the pool's mapped, unused memory

template <class T>
T *dmalloc(size_t count, cudaStream_t s) {
    if (count == 0) count = 1;
    void *p = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&p, count * sizeof(T), device_pool(), s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(PAIR_ERR_OOM, std::string("device allocation of ") + std::to_string(count * sizeof(T)) +
                               " bytes failed: " + cudaGetErrorString(e));
    }
    return static_cast<T *>(p);
}
inline void dfree(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// Lets kernel 'kern' take up to the device's opt-in shared memory per block.  The
// attribute belongs to the function, not to a launch: every caller sets the same
// maximal value, so hierarchies set up at the same time on several host threads
// cannot lower it under one another's launch.
template <class F>
void allow_max_dyn_smem(F kern) {
    int dev = 0, optin = 0;
    PR_CUDA(cudaGetDevice(&dev));
    PR_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    PR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
}

// Programmatic dependent launch: the kernel may start while the previous kernel
// on the stream finishes; it must begin with pdl_begin() (device side), which waits
// for the previous grid's completion and memory, then lets the next kernel launch.
template <typename... KArgs, typename... Args>
void launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cuda_check(cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...), "kernel launch", __FILE__, __LINE__);
}

#ifdef __CUDACC__
__device__ __forceinline__ void pdl_begin() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
#endif

#ifdef __CUDACC__
// |x| as an ordered integer key: for non-NaN doubles the bit patterns of |x|
// order exactly as the values, so pivot searches and maxima of magnitudes run
// on the integer pipe instead of the (narrow) FP64 pipe.
__device__ __forceinline__ long long absbits(double x) { return __double_as_longlong(x) & 0x7fffffffffffffffLL; }
#endif

// Exclusive scan of int counts (n entries) into out (n+1 entries, out[n] = total);
// returns the total (synchronises the stream).
long long scan_exclusive(const int *in, int *out, int n, cudaStream_t s, bool want_total = true);
// in place: v[0..n) becomes its exclusive prefix sums, v[n] (and the return) the total
long long scan_exclusive_ll(long long *v, int n, cudaStream_t s);

// ---------------------------------------------------------------------------
// Hierarchy storage.  A hierarchy holds a batch of independent matrices
// ("directions"); level l stores the concatenation of the level-l operators of
// every matrix that has a level l, in matrix order.
// ---------------------------------------------------------------------------
enum : int8_t { CF_F = 0, CF_C = 1, CF_COARSEST = 2 };

// Sliced ELL copy of a set of rows (32 rows per slice, rows ordered by decreasing
// length inside windows of 256): position q holds row[q] (-1: empty) with len[q]
// entries at ptr[q / 32] + (q % 32) + 32 j, j < len[q]
struct Sell {
    int nrows = 0, npos = 0;
    long long nnz = 0;   // stored slots including padding
    int *ptr = nullptr, *row = nullptr, *len = nullptr, *col = nullptr;
    short *col16 = nullptr;   // instead of col: column minus row, when every entry fits 16 bits
    void *val = nullptr;
    int G = 0;           // lanes per row chosen by the autotuner (0: size heuristic)
};

struct Level {
    int n = 0;
    long long nnz = 0;
    int *rowptr = nullptr, *col = nullptr;
    double *val = nullptr;
    double *dinv = nullptr;
    float *dinv32 = nullptr;
    int8_t *cf = nullptr;     // CF_F / CF_C / CF_COARSEST
    int *pmap = nullptr;      // P column per row (coarse index) or -1
    int *rowdir = nullptr;    // matrix slot of each row
    int nc = 0;
    int *cpts = nullptr;      // fine row of every coarse point
    int *zrowptr = nullptr, *zcol = nullptr;
    double *zval = nullptr;
    long long nnzZ = 0;
    // per matrix slot (host): first row, rows, coarse points, coarsest flag, stats
    std::vector<int> row0, nrows, ncdir, nnzdir, nnzZdir, singular;
    std::vector<char> coarsest;
    int pmis_rounds = 0;
    int *d_row0 = nullptr;    // device copy of row0 (size ndir)
    // coarsest segments (device): first row and rows of each matrix that ends here
    int n_cseg = 0;
    int *d_cseg_row0 = nullptr, *d_cseg_n = nullptr;
    // CF split for the V-cycle: srow lists the rows in the order [F | C | coarsest],
    // ascending within each group; sF, sC: SELL copies of the F and C rows, sZ of Z
    // (values in the cycle precision); sptr/scol/sval: CSR copy of the coarsest rows
    // in split order, d_cseg_s0: each coarsest segment's first position in it; sX:
    // SELL copy of the coarsest rows, built when a coarsest segment is too large for
    // the one-CTA shared-memory sweeps (its Jacobi sweeps then run grid-wide)
    int nF = 0, nC = 0;
    int *srow = nullptr, *sptr = nullptr, *scol = nullptr;
    void *sval = nullptr;
    int *d_cseg_s0 = nullptr;
    Sell sF, sC, sZ, sX;
    // V-cycle work vectors (precision of the hierarchy); vF is the buffer (vy or vxn)
    // that holds the F rows after the last F sweep, C rows are then in vx
    void *vb = nullptr, *vx = nullptr, *vxn = nullptr, *vy = nullptr;
    void *vF = nullptr;
};

// Level schedule of an exact sweep of a block-scaled upwind operator (sweep_dag.cu):
// single elements grouped by upwind level, and the cyclic components (strongly
// connected sets of at most SD_MAXE elements, solved as dense blocks) per level.
constexpr int SD_MAXE = 8;

// Shared memory of the one-CTA coarsest-level sweeps: a coarsest segment whose
// entries (value + column), four vectors and row pointer fit is swept in shared
// memory; a level with a larger one gets a SELL copy of its coarsest rows instead.
constexpr int CS_SMEM = 40 * 1024;
struct SweepPlan {
    int nb = 0, nlev = 0, ncomp = 0;
    int *list = nullptr;                     // single elements, level by level
    int *comp = nullptr, *compn = nullptr;   // component members (SD_MAXE per row) and sizes
    std::vector<long long> off;              // list offsets per level (nlev + 1)
    std::vector<int> comp_off;               // component-table offsets per level (nlev + 1)
    void release(cudaStream_t s);
};

// CUDA events of one V-cycle (also recorded inside captured graphs): the level-0
// relaxation, the FP32 inner residual, and the relaxation of every coarse level
// (2 per level); one slot per cycle position of a graph
struct ProfSlot {
    cudaEvent_t relax0[2] = {nullptr, nullptr};
    cudaEvent_t res32[2] = {nullptr, nullptr};
    std::vector<cudaEvent_t> lv;
    std::vector<cudaEvent_t> lvx;   // grid-wide coarsest sweeps of a level (2 per level)
    std::vector<cudaEvent_t> lvt;   // a level's restriction and prolongation (4 per level)
    bool relax_timed = false;   // relax0 recorded by the cycle
    bool res_timed = false;     // res32 recorded by the cycle
};

// A step's inner iteration of matrix m stops once its FP32 residual is at most
// max(INNER_TOL_FRAC tol ||b||, INNER_ETA ||r||), r the step's outer residual: no
// deeper than an FP32 iteration resolves in one step (the FP32 rounding of r32 - A d
// is ~1e-7 ||r||); the next step continues from the new outer residual.  From the
// second step on ||r|| <= tol ||b|| / INNER_ETA, so that rounding is at most
// 1e-7 / INNER_ETA = 1% of tol ||b|| and the inner estimate decides the outer test.
constexpr double INNER_TOL_FRAC = 1.0;
constexpr double INNER_ETA = 1e-5;

// cycle positions of the inner-cycle graphs: graph g runs 2^g cycles, on the
// slots [2^g - 1, 2^(g+1) - 1)
constexpr int INNER_GRAPHS = 5;
constexpr int INNER_SLOTS = (1 << INNER_GRAPHS) - 1;

// Captured graphs of a hierarchy's solve loop.
struct CycleGraphs {
    cudaGraphExec_t gcyc[INNER_GRAPHS] = {};      // 2^g inner cycles
    long long gcyc_kernels[INNER_GRAPHS] = {};
    cudaGraphExec_t gclose = nullptr;             // x += d, outer residual and norms
    long long gclose_kernels = 0;
    const double *gi_b = nullptr;
    double *gi_x = nullptr;
    double gi_tol = -1;
    cudaGraphExec_t graph = nullptr;              // one V-cycle + residual (or a sweep)
    long long graph_kernels = 0;
    const double *graph_b = nullptr;
    double *graph_x = nullptr;
    double graph_tol = -1;
    CycleGraphs() = default;
    CycleGraphs(const CycleGraphs &) = delete;
    CycleGraphs &operator=(const CycleGraphs &) = delete;
    ~CycleGraphs() {
        if (graph) cudaGraphExecDestroy(graph);
        for (auto &g : gcyc)
            if (g) cudaGraphExecDestroy(g);
        if (gclose) cudaGraphExecDestroy(gclose);
    }
};

struct Hier {
    int ndir = 0;
    air_params prm{};
    cudaStream_t stream = nullptr;   // private stream
    std::vector<int> n0;             // rows per matrix at level 0
    std::vector<Level> lev;
    // Level-0 block form of the structured hex operator (set by the SI driver)
    bool bsr0 = false;
    int hex_n = 0;
    double *bsr64 = nullptr;  // [dir][elem][axis][row a][4]
    float *bsr32 = nullptr;
    // FP32-refined block form: the outer residual in double-float arithmetic (pairs
    // of floats, hi + lo) instead of the FP64 pipe; block values, b and the solve's
    // iterate are held as pairs during a solve (bsr64 is then not kept)
    // FP32 relaxation of the block form on CF-split copies: v0[k] holds the three
    // face rows (float4 each) of the row at split position k of level 0 (F rows,
    // then C rows, as lev[0].srow); bsr32 is then not kept
    bool split0 = false;
    float4 *v0 = nullptr;
    bool dd = false;
    float2 *bsr_dd = nullptr;          // same layout as bsr64
    float2 *b_dd = nullptr, *x_dd = nullptr;   // [rows of the batch]
    int8_t *dsign = nullptr;  // [dir][3] sign of Omega components
    // solve state
    double *partials = nullptr;  // [dir][max blocks]
    int maxblk = 0;
    double *rnorm = nullptr, *bnorm = nullptr, *rnorm0 = nullptr;  // [dir]
    int *active = nullptr;                                         // [dir]
    int *d_err = nullptr;
    int *d_n0 = nullptr, *d_row00 = nullptr;  // level-0 rows per matrix and first rows
    int sms = 1;                              // multiprocessors of the device
    // FP32 inner correction (precision >= 1, solves with tol > 0): a refinement
    // step casts the outer residual r into r32 and iterates A d = r in FP32, each
    // inner cycle a V-cycle on the current inner residual (its correction added to
    // d32) followed by the FP32 residual r32 - A d32 and its norm; the step ends
    // with x += d and a new outer residual.  A matrix stops cycling (iactive = 0)
    // once its inner residual is at most ithr, set by the outer residual.
    bool inner = false;
    float *r32 = nullptr, *d32 = nullptr;        // [rows of the batch]
    float *val32 = nullptr;                       // CSR level 0 values in FP32
    int *iactive = nullptr, *icount = nullptr;    // [dir]: inner flag, cycles this step
    int *iany = nullptr;                          // 1 while a matrix of the batch still cycles
    unsigned *iticket = nullptr;                  // CTA ticket of the norm kernels (0 between launches)
    double *ithr = nullptr, *inorm = nullptr;     // [dir]
    double rho_est = 0.0;                         // contraction of the inner cycles (0: none yet)
    // captured graphs, one set without and one with the timing events (an event
    // between two kernels ends their programmatic overlap, so untimed solves replay
    // graphs without them)
    CycleGraphs gr[2];
    CycleGraphs &graphs() { return gr[timed ? 1 : 0]; }
    // instrumentation: CUDA events around the level-0 kernels and the coarse levels
    // (also inside graphs); ev[0..1] bracket the outer residual.  prof: the events
    // exist; timed: the current solve records them
    bool prof = false, timed = false;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    std::vector<ProfSlot> slots;       // slot 0: the per-cycle path; 0..INNER_SLOTS-1: inner graphs
    double t_res0 = 0, t_relax0 = 0, gb_res0 = 0, gb_relax0 = 0, t_res32 = 0, gb_res32 = 0;
    long long n_res0 = 0, n_relax0 = 0, n_res32 = 0;
    // per matrix: level-0 algorithmic bytes of one outer residual, one F+C relaxation
    // pass and one FP32 inner residual
    std::vector<double> bytes_res0, bytes_relax0, bytes_res32;
    double t_phase[4] = {0, 0, 0, 0};   // setup: strength+PMIS, P+lAIR, RAP, other
    // coarse-level (l >= 1) relaxation: bytes per cycle
    double t_relaxc = 0, gb_relaxc = 0, bytes_relaxc = 0;
    double t_relaxc_level[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // by level (entry k: level k + 1)
    long long n_relaxc = 0;
    // grid transfers (every level's restriction and prolongation): bytes per cycle
    double t_xfer = 0, gb_xfer = 0, bytes_xfer = 0;
    long long n_xfer = 0;
    SweepPlan *dag = nullptr;   // exact-sweep schedule of an unstructured batch
    ~Hier();
};

// setup.cu
void build_hierarchy(Hier &h);   // levels from lev[0] (CSR FP64), on h.stream
void free_level(Level &L, cudaStream_t s);

// cycle.cu
// r = b - A0 x (FP64), cast into lev[0].vb; per-matrix ||r||; active[d] = ||r|| > tol ||b||
// zero_x: x is known to be zero (r = b; the operator is not read, the launch not timed)
void residual0(Hier &h, const double *b, const double *x, double tol, bool update_active, bool zero_x = false);
void vcycle_correct(Hier &h, double *x, ProfSlot *ps = nullptr);   // x += V(lev[0].vb), zero initial guess
// inner correction (h.inner): outer residual into lev[0].vb and r32 with the norms,
// active and inner flags and thresholds; one inner cycle (V-cycle into d32, FP32
// residual and inner norm); x += d32 (d32 cleared) for the active matrices
void inner_enable(Hier &h);
void residual_outer(Hier &h, const double *b, const double *x, double tol, bool zero_x = false);
void inner_cycle(Hier &h, ProfSlot *ps);
void fold_delta(Hier &h, double *x);
// double-float mode (h.dd): b and x to pairs before a solve, x back after it; the
// residual and the final relaxation then work on h.b_dd / h.x_dd
void dd_enable(Hier &h);            // bsr_dd from bsr64 (frees bsr64), vectors
void split0_enable(Hier &h);        // v0 from bsr32 (frees bsr32)
void dd_load(Hier &h, const double *b, const double *x);
void dd_store(Hier &h, double *x);
void norms0(Hier &h, const double *v, double *out);  // per-matrix 2-norms of a level-0 vector
void alloc_cycle_vectors(Hier &h);
void set_all_active(Hier &h);   // every matrix of the batch takes part in the next cycle
void level0_bytes(Hier &h);   // fills bytes_res0 / bytes_relax0 (hex block form), bytes_relaxc
void prof_enable(Hier &h);
void autotune_cycle(Hier &h);   // lanes per row of every SELL kernel (timed once per shape)

// sweep.cu: x = A^{-1} b for every matrix of a batch: upwind wavefronts on a
// structured-hex batch with its block form (bsr64), otherwise the batch's level
// schedule (h.dag, sweep_dag.cu); graph-captured when use_graph
void sweep_solve(Hier &h, const double *b, double *x, bool use_graph);

// sweep_dag.cu: the level schedule of nd matrices of N rows each (nb DOFs per
// element, identity diagonal blocks) stacked block-diagonally in one CSR
// (global column indices), on stream s; the launches of one exact solve
SweepPlan *sweep_plan_build(int nd, long long N, int nb, const int *rowptr, const int *col, int *d_err,
                            cudaStream_t s);
void sweep_plan_launch(const SweepPlan &P, const int *rowptr, const int *col, const double *val, const double *b,
                       double *x, int *d_err, cudaStream_t s);
// plan, solve and release for one CSR matrix (synchronises s)
void sweep_csr(int n, int nb, const int *rowptr, const int *col, const double *val, const double *b, double *x,
               cudaStream_t s, int *ncomp, int *nlev);

// assemble.cu
void hex_assemble(int n, int ndir, const double *omega_d, const double *sigma_t, int *rowptr, int *col,
                  double *val, double *bsr64, float *bsr32, double *W, double *Gin, int *d_err, cudaStream_t s);
long long hex_nnz(int n, const double *omega_h);
long long tet_assemble(int T, int ndir, const double *omega_d, const double *verts, const int *tets, const int *nbr,
                       const double *sigma_t, int *rowptr, int *col, double *val, double *W, double *Gin, int *d_err,
                       cudaStream_t s, bool rowptr_only);

// si.cu
struct BatchSolve {
    bool converged = true;
    int iters = 0;          // V-cycles of the slowest matrix
    long long cycles = 0;   // V-cycles summed over the matrices
    int outer = 0;          // outer (FP64 / double-float) residuals taken
    double max_rel = 0;
    double rho_sum = 0;
    int rho_cnt = 0;
};
// x_zero: x holds zeros on entry (the first residual is then b itself)
BatchSolve solve_batch(Hier &h, const double *b, double *x, double tol, int maxit, bool use_graph,
                       bool x_zero = false);
void si_run(const pair_mesh &mesh, const pair_quad &quad, const double *sigma_t, const double *sigma_s,
            const double *q, const air_params &prm, const si_params &sp, double *phi, double *psi,
            cudaStream_t user, si_info *info);
void si_adjoint_run(const pair_mesh &mesh, const pair_quad &quad, const double *sigma_t, const double *sigma_s,
                    const double *psi, const double *g, const air_params &prm, const si_params &sp, double *dst,
                    double *dss, double *dq, double *phis_out, cudaStream_t user, si_info *info);
void csr_transpose_dev(int n, long long nnz, const int *rowptr, const int *col, const double *val, int *trp,
                       int *tcol, double *tval, cudaStream_t s);

}  // namespace pr
