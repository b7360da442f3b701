// Bottom of the AIR V-cycle (Sec. 1.2) in one launch: one thread-block cluster
// per matrix of the batch runs that matrix's restrictions, coarsest Jacobi sweeps,
// prolongations and F-F-C relaxations on every level from lb down, with cluster
// barriers between the steps instead of kernel boundaries.
//
// On the small levels of a hierarchy a sweep is a few thousand rows per matrix:
// as separate launches each step costs its launch and ramp time (5-8 us) however
// little it moves.  The matrices of a batch are independent, so each cluster
// owns one matrix and needs no grid-wide synchronisation.  The arithmetic and the
// order of the steps are those of the multi-launch cycle in cycle.cu: the same
// Jacobi sweeps on the CF-split rows, the same one-point prolongation and
// R = [Z, I] restriction (G = 4 lanes per row).
//
// Values written inside the kernel are read with ld.global.cg (L2, no L1 copy),
// and every step ends with a fence and a cluster barrier (release / acquire at
// cluster scope), so a CTA never reads another CTA's stale data.  Control flow
// around the barriers depends only on the matrix and the level, never on the
// thread, so every thread of the cluster reaches every barrier.
#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace pr {

namespace {

constexpr int BOT_CLUSTER = 8;     // CTAs per matrix (portable cluster size)
constexpr int BOT_BS = 256;
constexpr int BOT_G = 4;           // lanes per row in row dot products
constexpr int BOT_MAX_ROWS = 8192; // levels whose every matrix has at most this many rows

template <class T>
struct BLev {
    const int *srow, *sptr, *scol;
    const T *sval, *dinv;
    const int8_t *cf;
    const int *pmap;
    const int *cpts, *zptr, *zcol;   // restriction to the next level (rows = its rows)
    const T *zval;
    T *vb, *vx, *vxn, *vy;
};

// one matrix on one level: rows [row0, row0 + n), split runs of its F and C rows,
// split position of its rows if the matrix ends here (-1 otherwise), and its rows
// on the next level [crow0, crow0 + cn)
struct BDir {
    int row0, n, f0, nf, c0, nc, x0, crow0, cn;
};

__device__ __forceinline__ void cluster_step() {
    __threadfence();
    cg::this_cluster().sync();
}

// sum over entries [p0, p1) of val[p] * v[col[p]], G lanes, lane g takes p0+g, p0+g+G, ...
template <class T>
__device__ __forceinline__ T bot_dot(int p0, int p1, int g, const int *col, const T *val, const T *v) {
    T acc = T(0);
    for (int p = p0 + g; p < p1; p += BOT_G) acc += __ldcs(val + p) * __ldcg(v + __ldcs(col + p));
#pragma unroll
    for (int o = BOT_G / 2; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o, BOT_G);
    return acc;
}

template <class T>
__global__ void __launch_bounds__(BOT_BS) k_bottom(int nlev, int ndir, const BLev<T> *lev, const BDir *bd,
                                                   const int *dirs, int fsweeps, int csweeps) {
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int d = dirs[blockIdx.x / BOT_CLUSTER];
    const int nthr = BOT_CLUSTER * BOT_BS;
    const int tid = rank * BOT_BS + threadIdx.x;
    const int g = threadIdx.x % BOT_G;
    const int grp = tid / BOT_G, ngrp = nthr / BOT_G;
    // rows handled by a G-lane group must keep whole groups inside a warp
    // (BOT_BS is a multiple of 32 and BOT_G divides 32)

    // down: restrict until the level where this matrix ends
    int lend = nlev - 1;
    for (int l = 0; l < nlev; ++l) {
        const BDir D = bd[l * ndir + d];
        if (D.x0 >= 0 || l == nlev - 1) { lend = l; break; }
        const BLev<T> &L = lev[l];
        const BLev<T> &C = lev[l + 1];
        for (int r0 = 0; r0 < D.cn; r0 += ngrp) {
            int r = r0 + grp;
            bool ok = r < D.cn;
            int ic = D.crow0 + (ok ? r : 0);
            // every lane calls bot_dot (its shuffles need the whole warp); lanes past
            // the last row take an empty range
            T acc = bot_dot<T>(ok ? L.zptr[ic] : 0, ok ? L.zptr[ic + 1] : 0, g, L.zcol, L.zval, L.vb);
            if (ok && g == 0) C.vb[ic] = acc + __ldcg(L.vb + L.cpts[ic]);
        }
        cluster_step();
    }
    // coarsest: Jacobi sweeps from zero on this matrix's rows, by the first CTA
    {
        const BDir D = bd[lend * ndir + d];
        const BLev<T> &L = lev[lend];
        if (rank == 0 && D.x0 >= 0) {
            for (int li = threadIdx.x; li < D.n; li += BOT_BS) L.vx[D.row0 + li] = T(0);
            __threadfence_block();
            __syncthreads();
            T *cur = L.vx, *nxt = L.vxn;
            for (int s = 0; s < csweeps; ++s) {
                for (int li = threadIdx.x; li < D.n; li += BOT_BS) {
                    int i = D.row0 + li, k = D.x0 + li;
                    T acc = T(0);
                    for (int p = L.sptr[k]; p < L.sptr[k + 1]; ++p) acc += L.sval[p] * __ldcg(cur + L.scol[p]);
                    nxt[i] = __ldcg(cur + i) + L.dinv[i] * (__ldcg(L.vb + i) - acc);
                }
                __threadfence_block();
                __syncthreads();
                T *t = cur; cur = nxt; nxt = t;
            }
            if (cur != L.vx)
                for (int li = threadIdx.x; li < D.n; li += BOT_BS) L.vx[D.row0 + li] = __ldcg(cur + D.row0 + li);
        }
        cluster_step();
    }
    // up: prolong, F sweeps, C sweep on every level above lend
    for (int l = lend - 1; l >= 0; --l) {
        const BDir D = bd[l * ndir + d];
        const BLev<T> &L = lev[l];
        const BLev<T> &C = lev[l + 1];
        const T *xcF = (fsweeps & 1) ? C.vxn : C.vy;   // F rows of the coarse level after its sweeps
        for (int li = tid; li < D.n; li += nthr) {
            int i = D.row0 + li;
            int8_t c = L.cf[i];
            if (c == CF_COARSEST) continue;
            int p = L.pmap[i];
            T v = T(0);
            if (p >= 0) v = C.cf[p] == CF_F ? __ldcg(xcF + p) : __ldcg(C.vx + p);
            L.vy[i] = v;
            if (c == CF_C) L.vxn[i] = v;
        }
        cluster_step();
        T *bufs[2] = {L.vy, L.vxn};
        int cur = 0;
        for (int f = 0; f < fsweeps; ++f, cur ^= 1) {
            const T *in = bufs[cur];
            T *out = bufs[cur ^ 1];
            for (int r0 = 0; r0 < D.nf; r0 += ngrp) {
                int r = r0 + grp;
                bool ok = r < D.nf;
                int k = D.f0 + (ok ? r : 0);
                T acc = bot_dot<T>(ok ? L.sptr[k] : 0, ok ? L.sptr[k + 1] : 0, g, L.scol, L.sval, in);
                if (ok && g == 0) {
                    int i = L.srow[k];
                    out[i] = __ldcg(in + i) + L.dinv[i] * (__ldcg(L.vb + i) - acc);
                }
            }
            cluster_step();
        }
        {
            const T *in = bufs[cur];
            for (int r0 = 0; r0 < D.nc; r0 += ngrp) {
                int r = r0 + grp;
                bool ok = r < D.nc;
                int k = D.c0 + (ok ? r : 0);
                T acc = bot_dot<T>(ok ? L.sptr[k] : 0, ok ? L.sptr[k + 1] : 0, g, L.scol, L.sval, in);
                if (ok && g == 0) {
                    int i = L.srow[k];
                    L.vx[i] = __ldcg(in + i) + L.dinv[i] * (__ldcg(L.vb + i) - acc);
                }
            }
            cluster_step();
        }
    }
}

template <class T>
const T *sval_of(const Level &L) { return (const T *)L.sval; }
template <class T>
const T *dinv_of(const Level &L);
template <>
const float *dinv_of<float>(const Level &L) { return L.dinv32; }
template <>
const double *dinv_of<double>(const Level &L) { return L.dinv; }
template <class T>
const T *zval_of(const Level &L);
template <>
const float *zval_of<float>(const Level &L) { return L.zval32; }
template <>
const double *zval_of<double>(const Level &L) { return L.zval; }

template <class T>
void upload_levels(Hier &h) {
    const int NL = (int)h.lev.size();
    std::vector<BLev<T>> v;
    for (int l = h.lb; l < NL; ++l) {
        const Level &L = h.lev[l];
        BLev<T> b{};
        b.srow = L.srow; b.sptr = L.sptr; b.scol = L.scol; b.sval = sval_of<T>(L); b.dinv = dinv_of<T>(L);
        b.cf = L.cf; b.pmap = L.pmap; b.cpts = L.cpts; b.zptr = L.zrowptr; b.zcol = L.zcol; b.zval = zval_of<T>(L);
        b.vb = (T *)L.vb; b.vx = (T *)L.vx; b.vxn = (T *)L.vxn; b.vy = (T *)L.vy;
        v.push_back(b);
    }
    h.d_blev = dmalloc<char>(sizeof(BLev<T>) * v.size(), h.stream);
    PR_CUDA(cudaMemcpyAsync(h.d_blev, v.data(), sizeof(BLev<T>) * v.size(), cudaMemcpyHostToDevice, h.stream));
    PR_CUDA(cudaStreamSynchronize(h.stream));
}

template <class T>
void launch_bottom(Hier &h) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(h.n_bdirs * BOT_CLUSTER), 1, 1);
    cfg.blockDim = dim3(BOT_BS, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = h.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = BOT_CLUSTER;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const int nlev = (int)h.lev.size() - h.lb;
    PR_CUDA(cudaLaunchKernelEx(&cfg, k_bottom<T>, nlev, h.ndir, (const BLev<T> *)h.d_blev, (const BDir *)h.d_bdir,
                               (const int *)h.d_bdirs, h.prm.f_sweeps, h.prm.coarse_sweeps));
    PR_LAUNCH();
}

}  // namespace

// Chooses lb (the first level from which every level has at most BOT_MAX_ROWS rows
// per matrix) and uploads the per-level pointers and per-matrix row ranges.
// lb = number of levels means no bottom kernel.
void bottom_prepare(Hier &h) {
    const int NL = (int)h.lev.size();
    const int ND = h.ndir;
    h.lb = NL;
    for (int l = NL - 1; l >= 1; --l) {
        const Level &L = h.lev[l];
        bool small = (int)L.nrows.size() == ND && L.srow != nullptr;
        for (int d = 0; d < ND && small; ++d) small = L.nrows[d] <= BOT_MAX_ROWS;
        if (!small) break;
        h.lb = l;
    }
    if (h.lb >= NL) return;
    // per (level, matrix) row ranges; F and C runs of a matrix are contiguous in
    // the split order because rows are matrix-major and each group is ascending
    std::vector<BDir> bd;
    for (int l = h.lb; l < NL; ++l) {
        const Level &L = h.lev[l];
        int f = 0, c = L.nF, x = L.nF + L.nC;
        for (int d = 0; d < ND; ++d) {
            BDir D{};
            D.row0 = L.row0[d];
            D.n = L.nrows[d];
            D.x0 = -1;
            if (D.n > 0 && L.coarsest[d]) {
                D.x0 = x;
                x += D.n;
            } else if (D.n > 0) {
                D.nc = L.ncdir[d];
                D.nf = D.n - D.nc;
                D.f0 = f;
                D.c0 = c;
                f += D.nf;
                c += D.nc;
            }
            if (l + 1 < NL && D.n > 0 && !L.coarsest[d]) {
                D.crow0 = h.lev[l + 1].row0[d];
                D.cn = h.lev[l + 1].nrows[d];
            }
            bd.push_back(D);
        }
        PR_REQUIRE(f == L.nF && c == L.nF + L.nC && x == L.n, PAIR_ERR_DEVICE,
                   "bottom cycle: per-matrix CF counts do not add up to the level's");
    }
    std::vector<int> dirs;
    for (int d = 0; d < ND; ++d)
        if (h.lev[h.lb].nrows[d] > 0) dirs.push_back(d);
    h.n_bdirs = (int)dirs.size();
    if (h.n_bdirs == 0) {
        h.lb = NL;
        return;
    }
    h.d_bdir = dmalloc<char>(sizeof(BDir) * bd.size(), h.stream);
    PR_CUDA(cudaMemcpyAsync(h.d_bdir, bd.data(), sizeof(BDir) * bd.size(), cudaMemcpyHostToDevice, h.stream));
    h.d_bdirs = dmalloc<int>(dirs.size(), h.stream);
    PR_CUDA(cudaMemcpyAsync(h.d_bdirs, dirs.data(), sizeof(int) * dirs.size(), cudaMemcpyHostToDevice, h.stream));
    if (h.prm.precision == 1) upload_levels<float>(h);
    else upload_levels<double>(h);
}

void bottom_cycle(Hier &h) {
    if (h.prm.precision == 1) launch_bottom<float>(h);
    else launch_bottom<double>(h);
}

}  // namespace pr
