// extern "C" boundary of libpair (declared in include/pair.h).  Every entry
// point converts internal errors into a pair_status and a per-thread message.
#include <algorithm>
#include <cstdio>
#include <cmath>
#include <cstring>

#include <type_traits>
#include <vector>

#include "common.cuh"


struct pair_hier_s {
    pr::Hier h;
};

namespace {

thread_local std::string g_last_error;

template <class F>
pair_status guarded(F &&f) {
    try {
        f();
        g_last_error.clear();
        return PAIR_OK;
    } catch (const pr::Error &e) {
        g_last_error = e.msg;
        return e.st;
    } catch (const std::bad_alloc &) {
        g_last_error = "host allocation failed";
        return PAIR_ERR_OOM;
    } catch (const std::exception &e) {
        g_last_error = e.what();
        return PAIR_ERR_CUDA;
    } catch (...) {
        g_last_error = "unknown internal error";
        return PAIR_ERR_CUDA;
    }
}

void check_params(const air_params *p) {
    PR_REQUIRE(p, PAIR_ERR_ARG, "air_params is null");
    PR_REQUIRE(p->distance == 1 || p->distance == 2, PAIR_ERR_ARG, "distance must be 1 or 2");
    PR_REQUIRE(p->theta > 0 && p->theta <= 1 && p->eps_R > 0 && p->eps_R <= 1, PAIR_ERR_ARG,
               "theta and eps_R must lie in (0, 1]");
    PR_REQUIRE(p->phi_R >= 0 && p->phi_R < 1 && p->phi_A >= 0 && p->phi_A < 1, PAIR_ERR_ARG,
               "phi_R and phi_A must lie in [0, 1)");
    PR_REQUIRE(p->max_levels >= 1 && p->max_coarse >= 1 && p->coarse_sweeps >= 0, PAIR_ERR_ARG,
               "max_levels, max_coarse must be >= 1 and coarse_sweeps >= 0");
    PR_REQUIRE(p->precision >= 0 && p->precision <= 2, PAIR_ERR_ARG,
               "precision must be 0 (FP64), 1 (FP32 cycle, FP64 refinement) or 2 (FP32 cycle, float-pair refinement)");
    PR_REQUIRE(p->f_sweeps >= 1 && p->f_sweeps <= 8, PAIR_ERR_ARG, "f_sweeps must lie in [1, 8]");
    PR_REQUIRE(p->nair == 0 || p->nair == 1, PAIR_ERR_ARG, "nair must be 0 (lAIR) or 1 (nAIR degree 1)");
}

__global__ void k_concat_rowptr(int n, const int *in, int *out, int off) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= n) out[i] = in[i] - in[0] + off;
}
__global__ void k_concat_col(int nnz, const int *in, int *out, int off) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nnz) out[i] = in[i] + off;
}
__global__ void k_fill_range(int *a, int n, int v) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

struct StreamJoin {
    // orders a private stream after the caller's stream and back
    cudaStream_t user, priv;
    cudaEvent_t ev;
    StreamJoin(cudaStream_t u, cudaStream_t p) : user(u), priv(p) {
        PR_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        PR_CUDA(cudaEventRecord(ev, user));
        PR_CUDA(cudaStreamWaitEvent(priv, ev, 0));
    }
    ~StreamJoin() {
        cudaEventRecord(ev, priv);
        cudaStreamWaitEvent(user, ev, 0);
        cudaEventDestroy(ev);
    }
};

}  // namespace

void pr::set_last_error(const std::string &msg) { g_last_error = msg; }

namespace {
// true for host memory (pinned, registered or pageable), false for memory a kernel
// can read (device or managed)
bool is_host_ptr(const void *p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}

// Device copies of the host arrays among a call's arguments: inputs copied in on
// the stream before the work, outputs copied back after it, staging freed at exit.
struct HostStage {
    cudaStream_t s;
    std::vector<void *> bufs;
    struct Out {
        void *host;
        const void *dev;
        size_t bytes;
    };
    std::vector<Out> outs;
    explicit HostStage(cudaStream_t st) : s(st) {}
    ~HostStage() {
        for (void *b : bufs) cudaFreeAsync(b, s);
        cudaStreamSynchronize(s);
    }
    template <class T>
    T *in(T *p, size_t count, bool copy_back = false) {
        if (!p || count == 0 || !is_host_ptr(p)) return p;
        auto *d = pr::dmalloc<std::remove_const_t<T>>(count, s);
        bufs.push_back(d);
        PR_CUDA(cudaMemcpyAsync(d, p, sizeof(T) * count, cudaMemcpyHostToDevice, s));
        if (copy_back) outs.push_back({(void *)p, d, sizeof(T) * count});
        return d;
    }
    template <class T>
    T *out(T *p, size_t count) {   // written by the call only
        if (!p || count == 0 || !is_host_ptr(p)) return p;
        auto *d = pr::dmalloc<std::remove_const_t<T>>(count, s);
        bufs.push_back(d);
        outs.push_back({(void *)p, d, sizeof(T) * count});
        return d;
    }
    void copy_back() {
        for (auto &o : outs) PR_CUDA(cudaMemcpyAsync(o.host, o.dev, o.bytes, cudaMemcpyDeviceToHost, s));
        PR_CUDA(cudaStreamSynchronize(s));
    }
};
}  // namespace

extern "C" {

void air_params_default(air_params *p) {
    if (!p) return;
    p->distance = 1;
    p->theta = 0.25;
    p->eps_R = 0.01;
    p->phi_R = 0.0;
    p->phi_A = 0.0;
    p->max_levels = 25;
    p->max_coarse = 100;
    p->coarse_sweeps = 20;
    p->seed = 3;
    p->precision = 1;
    p->f_sweeps = 2;
    p->nair = 0;
}

void si_params_default(si_params *p) {
    if (!p) return;
    p->tol = 1e-8;
    p->max_iters = 500;
    p->inner_tol = 1e-8;
    p->inner_maxit = 100;
    p->batch = 0;
    p->mem_budget_gb = 0;
    p->g_inflow = 0;
    p->use_graphs = 1;
    p->fixed_iters = 0;
    p->solver = 0;
    p->inner_cycles = 0;
    p->q_ang = nullptr;
    p->phi_reduce = nullptr;
    p->reduce_ctx = nullptr;
    p->concurrent = 0;
    p->timing = 0;
}

const char *pair_last_error(void) { return g_last_error.c_str(); }

long long pair_kernel_launches(void) { return pr::g_launches; }

pair_status air_setup(const pair_csr *A, int count, const air_params *prm, void *stream, pair_hier *out) {
    return guarded([&] {
        PR_REQUIRE(A && out && count >= 1, PAIR_ERR_ARG, "air_setup: null argument or count < 1");
        check_params(prm);
        *out = nullptr;
        long long ntot = 0, nnztot = 0;
        for (int d = 0; d < count; ++d) {
            PR_REQUIRE(A[d].n >= 1 && A[d].nnz >= 0 && A[d].rowptr && (A[d].nnz == 0 || (A[d].col && A[d].val)),
                       PAIR_ERR_ARG, "air_setup: matrix " + std::to_string(d) + " has a null array or n < 1");
            ntot += A[d].n;
            nnztot += A[d].nnz;
        }
        PR_REQUIRE(ntot < 0x7fffffffLL && nnztot < 0x7fffffffLL, PAIR_ERR_UNSUPPORTED,
                   "air_setup: batch exceeds 2^31 rows or entries");
        auto *hh = new pair_hier_s;
        pr::Hier &h = hh->h;
        try {
            PR_CUDA(cudaStreamCreateWithFlags(&h.stream, cudaStreamNonBlocking));
            cudaStream_t s = h.stream;
            {
                StreamJoin join((cudaStream_t)stream, s);
                h.ndir = count;
                h.prm = *prm;
                h.d_err = pr::dmalloc<int>(1, s);
                PR_CUDA(cudaMemsetAsync(h.d_err, 0, sizeof(int), s));
                h.lev.resize(1);
                pr::Level &L = h.lev[0];
                L.n = (int)ntot;
                L.nnz = nnztot;
                L.rowptr = pr::dmalloc<int>(ntot + 1, s);
                L.col = pr::dmalloc<int>(nnztot, s);
                L.val = pr::dmalloc<double>(nnztot, s);
                L.rowdir = pr::dmalloc<int>(ntot, s);
                L.row0.resize(count);
                L.nrows.resize(count);
                h.n0.resize(count);
                int r = 0, z = 0;
                for (int d = 0; d < count; ++d) {
                    int n = A[d].n, nnz = A[d].nnz;
                    k_concat_rowptr<<<pr::blocks_for(n + 1, 256), 256, 0, s>>>(n, A[d].rowptr, L.rowptr + r, z);
                    PR_LAUNCH();
                    if (nnz) {
                        k_concat_col<<<pr::blocks_for(nnz, 256), 256, 0, s>>>(nnz, A[d].col, L.col + z, r);
                        PR_LAUNCH();
                        PR_CUDA(cudaMemcpyAsync(L.val + z, A[d].val, sizeof(double) * nnz, cudaMemcpyDeviceToDevice, s));
                    }
                    k_fill_range<<<pr::blocks_for(n, 256), 256, 0, s>>>(L.rowdir + r, n, d);
                    PR_LAUNCH();
                    L.row0[d] = r;
                    L.nrows[d] = n;
                    h.n0[d] = n;
                    r += n;
                    z += nnz;
                }
                L.d_row0 = pr::dmalloc<int>(count, s);
                h.d_row00 = pr::dmalloc<int>(count, s);
                h.d_n0 = pr::dmalloc<int>(count, s);
                PR_CUDA(cudaMemcpyAsync(L.d_row0, L.row0.data(), sizeof(int) * count, cudaMemcpyHostToDevice, s));
                PR_CUDA(cudaMemcpyAsync(h.d_row00, L.row0.data(), sizeof(int) * count, cudaMemcpyHostToDevice, s));
                PR_CUDA(cudaMemcpyAsync(h.d_n0, h.n0.data(), sizeof(int) * count, cudaMemcpyHostToDevice, s));
                pr::build_hierarchy(h);
                pr::alloc_cycle_vectors(h);
                pr::inner_enable(h);
                PR_CUDA(cudaStreamSynchronize(s));
            }
        } catch (...) {
            delete hh;
            throw;
        }
        *out = hh;
    });
}

pair_status air_vcycle(pair_hier hh, const double *b, double *x, void *stream) {
    return guarded([&] {
        PR_REQUIRE(hh && b && x, PAIR_ERR_ARG, "air_vcycle: null argument");
        pr::Hier &h = hh->h;
        StreamJoin join((cudaStream_t)stream, h.stream);
        pr::set_all_active(h);
        pr::residual0(h, b, x, 0.0, false);
        pr::vcycle_correct(h, x);
    });
}

pair_status air_solve(pair_hier hh, const double *b, double *x, double tol, int maxit, void *stream,
                      air_solve_info *info) {
    return guarded([&] {
        PR_REQUIRE(hh && b && x && tol >= 0 && maxit >= 0, PAIR_ERR_ARG, "air_solve: bad argument");
        pr::Hier &h = hh->h;
        PR_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
        pr::BatchSolve bs = pr::solve_batch(h, b, x, tol, maxit, false);
        PR_CUDA(cudaStreamSynchronize(h.stream));
        if (info) {
            info->iters = bs.iters;
            info->rel_resid = bs.max_rel;
            info->rho = bs.rho_cnt ? bs.rho_sum / bs.rho_cnt : 0.0;
        }
        if (!bs.converged) {
            char buf[160];
            snprintf(buf, sizeof buf, "air_solve: %d cycles, relative residual %.3e > %.3e", bs.iters, bs.max_rel,
                     tol);
            pr::fail(PAIR_ERR_NOT_CONVERGED, buf);
        }
    });
}

pair_status air_hier_nlevels(pair_hier hh, int mat, int *nlevels) {
    return guarded([&] {
        PR_REQUIRE(hh && nlevels, PAIR_ERR_ARG, "air_hier_nlevels: null argument");
        pr::Hier &h = hh->h;
        PR_REQUIRE(mat >= 0 && mat < h.ndir, PAIR_ERR_ARG, "air_hier_nlevels: matrix index out of range");
        int c = 0;
        for (auto &L : h.lev)
            if ((int)L.nrows.size() > mat && L.nrows[mat] > 0) ++c;
        *nlevels = c;
    });
}

pair_status air_level_info(pair_hier hh, int mat, int level, pair_level_info *out) {
    return guarded([&] {
        PR_REQUIRE(hh && out, PAIR_ERR_ARG, "air_level_info: null argument");
        pr::Hier &h = hh->h;
        PR_REQUIRE(mat >= 0 && mat < h.ndir && level >= 0 && level < (int)h.lev.size() &&
                       h.lev[level].nrows[mat] > 0,
                   PAIR_ERR_ARG, "air_level_info: no such level");
        const pr::Level &L = h.lev[level];
        out->n = L.nrows[mat];
        out->nnz = L.nnzdir[mat];
        out->coarsest = L.coarsest[mat] ? 1 : 0;
        out->nc = out->coarsest ? 0 : L.ncdir[mat];
        out->nnz_R = out->coarsest ? 0 : L.nnzZdir[mat];
        out->pmis_rounds = L.pmis_rounds;
        out->n_singular = L.singular[mat];
    });
}

pair_status air_level_export(pair_hier hh, int mat, int level, int *rowptr, int *col, double *val, signed char *cf,
                             int *pmap, int *cpts, int *zrowptr, int *zcol, double *zval) {
    return guarded([&] {
        PR_REQUIRE(hh, PAIR_ERR_ARG, "air_level_export: null handle");
        pr::Hier &h = hh->h;
        PR_REQUIRE(mat >= 0 && mat < h.ndir && level >= 0 && level < (int)h.lev.size() &&
                       h.lev[level].nrows[mat] > 0,
                   PAIR_ERR_ARG, "air_level_export: no such level");
        cudaStream_t s = h.stream;
        PR_CUDA(cudaStreamSynchronize(s));
        const pr::Level &L = h.lev[level];
        int r0 = L.row0[mat], n = L.nrows[mat];
        std::vector<int> rp(n + 1);
        PR_CUDA(cudaMemcpy(rp.data(), L.rowptr + r0, sizeof(int) * (n + 1), cudaMemcpyDeviceToHost));
        int p0 = rp[0], nnz = rp[n] - rp[0];
        if (rowptr)
            for (int i = 0; i <= n; ++i) rowptr[i] = rp[i] - p0;
        if (col) {
            PR_CUDA(cudaMemcpy(col, L.col + p0, sizeof(int) * nnz, cudaMemcpyDeviceToHost));
            for (int k = 0; k < nnz; ++k) col[k] -= r0;
        }
        if (val) PR_CUDA(cudaMemcpy(val, L.val + p0, sizeof(double) * nnz, cudaMemcpyDeviceToHost));
        if (L.coarsest[mat]) return;
        const pr::Level &C = h.lev[level + 1];
        int c0 = C.row0[mat], nc = L.ncdir[mat];
        if (cf) PR_CUDA(cudaMemcpy(cf, L.cf + r0, n, cudaMemcpyDeviceToHost));
        if (pmap) {
            PR_CUDA(cudaMemcpy(pmap, L.pmap + r0, sizeof(int) * n, cudaMemcpyDeviceToHost));
            for (int i = 0; i < n; ++i)
                if (pmap[i] >= 0) pmap[i] -= c0;
        }
        if (cpts) {
            PR_CUDA(cudaMemcpy(cpts, L.cpts + c0, sizeof(int) * nc, cudaMemcpyDeviceToHost));
            for (int i = 0; i < nc; ++i) cpts[i] -= r0;
        }
        std::vector<int> zr(nc + 1);
        PR_CUDA(cudaMemcpy(zr.data(), L.zrowptr + c0, sizeof(int) * (nc + 1), cudaMemcpyDeviceToHost));
        int z0 = zr[0], nz = zr[nc] - zr[0];
        if (zrowptr)
            for (int i = 0; i <= nc; ++i) zrowptr[i] = zr[i] - z0;
        if (zcol) {
            PR_CUDA(cudaMemcpy(zcol, L.zcol + z0, sizeof(int) * nz, cudaMemcpyDeviceToHost));
            for (int k = 0; k < nz; ++k) zcol[k] -= r0;
        }
        if (zval) PR_CUDA(cudaMemcpy(zval, L.zval + z0, sizeof(double) * nz, cudaMemcpyDeviceToHost));
    });
}

void air_free(pair_hier hh) { delete hh; }

static void check_mesh(const pair_mesh *mesh, const char *who) {
    PR_REQUIRE(mesh, PAIR_ERR_ARG, std::string(who) + ": null mesh");
    if (mesh->kind == PAIR_MESH_HEX) {
        PR_REQUIRE(mesh->n >= 1, PAIR_ERR_ARG, std::string(who) + ": hex mesh needs n >= 1");
    } else {
        PR_REQUIRE(mesh->kind == PAIR_MESH_TET && mesh->ntet >= 1 && mesh->verts && mesh->tets && mesh->nbr,
                   PAIR_ERR_ARG, std::string(who) + ": tet mesh needs ntet >= 1 and verts, tets, nbr");
    }
}

pair_status dg_assemble_tet(const pair_mesh *mesh, const double *omega, const double *sigma_t, int *rowptr, int *col,
                            double *val, int capacity, int *nnz, void *stream) {
    return guarded([&] {
        check_mesh(mesh, "dg_assemble_tet");
        PR_REQUIRE(mesh->kind == PAIR_MESH_TET && omega && sigma_t && rowptr && nnz, PAIR_ERR_ARG,
                   "dg_assemble_tet: bad argument");
        cudaStream_t s = (cudaStream_t)stream;
        double *om = pr::dmalloc<double>(3, s);
        int *err = pr::dmalloc<int>(1, s);
        PR_CUDA(cudaMemcpyAsync(om, omega, 3 * sizeof(double), cudaMemcpyHostToDevice, s));
        PR_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
        long long z = pr::tet_assemble(mesh->ntet, 1, om, mesh->verts, mesh->tets, mesh->nbr, sigma_t, rowptr,
                                       nullptr, nullptr, nullptr, nullptr, err, s, true);
        *nnz = (int)z;
        if (col && val && capacity >= z)
            pr::tet_assemble(mesh->ntet, 1, om, mesh->verts, mesh->tets, mesh->nbr, sigma_t, rowptr, col, val,
                             nullptr, nullptr, err, s, false);
        int herr = 0;
        PR_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
        PR_CUDA(cudaStreamSynchronize(s));
        pr::dfree(om, s);
        pr::dfree(err, s);
        PR_REQUIRE(herr == 0, PAIR_ERR_SINGULAR, "dg_assemble_tet: degenerate tetrahedron or face mismatch");
    });
}

pair_status dg_hex_nnz(const pair_mesh *mesh, const double *omega, int *nnz) {
    return guarded([&] {
        PR_REQUIRE(mesh && omega && nnz && mesh->kind == PAIR_MESH_HEX && mesh->n >= 1, PAIR_ERR_ARG,
                   "dg_hex_nnz: bad argument");
        long long v = pr::hex_nnz(mesh->n, omega);
        PR_REQUIRE(v < 0x7fffffffLL, PAIR_ERR_UNSUPPORTED, "dg_hex_nnz: more than 2^31 entries");
        *nnz = (int)v;
    });
}

pair_status dg_assemble_hex(const pair_mesh *mesh, const double *omega, const double *sigma_t, int *rowptr, int *col,
                            double *val, void *stream) {
    return guarded([&] {
        PR_REQUIRE(mesh && omega && sigma_t && rowptr && col && val && mesh->kind == PAIR_MESH_HEX && mesh->n >= 1,
                   PAIR_ERR_ARG, "dg_assemble_hex: bad argument");
        PR_REQUIRE(std::isfinite(omega[0]) && std::isfinite(omega[1]) && std::isfinite(omega[2]), PAIR_ERR_ARG,
                   "dg_assemble_hex: non-finite direction");
        cudaStream_t s = (cudaStream_t)stream;
        double *om = pr::dmalloc<double>(3, s);
        int *err = pr::dmalloc<int>(1, s);
        PR_CUDA(cudaMemcpyAsync(om, omega, 3 * sizeof(double), cudaMemcpyHostToDevice, s));
        PR_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
        pr::hex_assemble(mesh->n, 1, om, sigma_t, rowptr, col, val, nullptr, nullptr, nullptr, nullptr, err, s);
        int herr = 0;
        PR_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
        PR_CUDA(cudaStreamSynchronize(s));
        pr::dfree(om, s);
        pr::dfree(err, s);
        PR_REQUIRE(herr == 0, PAIR_ERR_SINGULAR, "dg_assemble_hex: singular element block");
    });
}


pair_status si_solve(const pair_mesh *mesh, const pair_quad *quad, const double *sigma_t, const double *sigma_s,
                     const double *q, const air_params *air, const si_params *sp, double *phi, double *psi,
                     void *stream, si_info *info) {
    return guarded([&] {
        PR_REQUIRE(quad && sigma_t && sigma_s && q && sp && phi, PAIR_ERR_ARG, "si_solve: null argument");
        check_mesh(mesh, "si_solve");
        PR_REQUIRE(quad->M >= 1 && quad->omega && quad->w, PAIR_ERR_ARG, "si_solve: empty quadrature");
        check_params(air);
        PR_REQUIRE(sp->tol >= 0 && sp->max_iters >= 1 && sp->inner_tol > 0 && sp->inner_maxit >= 1, PAIR_ERR_ARG,
                   "si_solve: bad si_params");
        PR_REQUIRE(sp->solver == 0 || sp->solver == 1, PAIR_ERR_ARG, "si_solve: solver must be 0 (AIR) or 1 (sweep)");
        PR_REQUIRE(sp->inner_cycles >= 0, PAIR_ERR_ARG, "si_solve: inner_cycles must be >= 0");
        for (int m = 0; m < quad->M; ++m)
            for (int k = 0; k < 3; ++k)
                PR_REQUIRE(std::isfinite(quad->omega[3 * m + k]) && std::isfinite(quad->w[m]), PAIR_ERR_ARG,
                           "si_solve: non-finite quadrature");
        // host arrays are staged through device copies on the caller's stream
        const bool hex = mesh->kind == PAIR_MESH_HEX;
        const size_t E = hex ? (size_t)mesh->n * mesh->n * mesh->n : (size_t)mesh->ntet, N = (hex ? 8 : 4) * E;
        const size_t M = (size_t)quad->M;
        HostStage st((cudaStream_t)stream);
        si_params spd = *sp;
        spd.q_ang = st.in(sp->q_ang, N * M);
        const double *dst = st.in(sigma_t, E), *dss = st.in(sigma_s, E), *dq = st.in(q, E);
        double *dphi = st.in(phi, N, true);
        double *dpsi = st.out(psi, N * M);
        pr::si_run(*mesh, *quad, dst, dss, dq, *air, spd, dphi, dpsi, (cudaStream_t)stream, info);
        st.copy_back();
    });
}

pair_status si_adjoint(const pair_mesh *mesh, const pair_quad *quad, const double *sigma_t, const double *sigma_s,
                       const double *q, const double *psi, const double *g, const air_params *air,
                       const si_params *sp, double *dJ_dsigma_t, double *dJ_dsigma_s, double *dJ_dq,
                       double *phi_adjoint, void *stream, si_info *info) {
    return guarded([&] {
        PR_REQUIRE(quad && sigma_t && sigma_s && q && psi && g && sp && dJ_dsigma_t && dJ_dsigma_s && dJ_dq,
                   PAIR_ERR_ARG, "si_adjoint: null argument");
        check_mesh(mesh, "si_adjoint");
        PR_REQUIRE(quad->M >= 1 && quad->omega && quad->w, PAIR_ERR_ARG, "si_adjoint: empty quadrature");
        check_params(air);
        PR_REQUIRE(sp->tol >= 0 && sp->max_iters >= 1 && sp->inner_tol > 0 && sp->inner_maxit >= 1, PAIR_ERR_ARG,
                   "si_adjoint: bad si_params");
        pr::si_adjoint_run(*mesh, *quad, sigma_t, sigma_s, psi, g, *air, *sp, dJ_dsigma_t, dJ_dsigma_s, dJ_dq,
                           phi_adjoint, (cudaStream_t)stream, info);
    });
}

pair_status pair_csr_transpose(const pair_csr *A, int *trowptr, int *tcol, double *tval, void *stream) {
    return guarded([&] {
        PR_REQUIRE(A && A->rowptr && trowptr && A->n >= 1 && A->nnz >= 0 &&
                       (A->nnz == 0 || (A->col && A->val && tcol && tval)),
                   PAIR_ERR_ARG, "pair_csr_transpose: bad argument");
        cudaStream_t s = (cudaStream_t)stream;
        pr::csr_transpose_dev(A->n, A->nnz, A->rowptr, A->col, A->val, trowptr, tcol, tval, s);
        PR_CUDA(cudaStreamSynchronize(s));
    });
}

pair_status pair_sweep(const pair_csr *A, int nb, const double *b, double *x, void *stream, int *n_cycles,
                       int *n_levels) {
    return guarded([&] {
        PR_REQUIRE(A && A->rowptr && A->col && A->val && b && x && A->n >= 1 && A->nnz >= 0 && (nb == 4 || nb == 8) &&
                       A->n % nb == 0,
                   PAIR_ERR_ARG, "pair_sweep: bad argument");
        pr::sweep_csr(A->n, nb, A->rowptr, A->col, A->val, b, x, (cudaStream_t)stream, n_cycles, n_levels);
    });
}

}  // extern "C"
