/*
 * CPU oracle for pAIR-in-source-iteration (Hanophy, Southworth, Li, Morel,
 * Manteuffel, "Parallel approximate ideal restriction multigrid for solving
 * the S_N transport equations").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, single-threaded FP64
 * restatement of what the GPU path computes, used by the tests, by smoke()
 * and by the benchmark's CPU-baseline leg.  The product library never links,
 * loads or calls it, and it shares no code with the CUDA sources.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no implicit FMA contraction,
 * so every product and sum is rounded exactly as written; the few fused
 * multiply-adds are explicit fma() calls).
 *
 * Contents (each function cites the passage it follows):
 *   - dense LU with partial pivoting (element blocks, lAIR local systems)
 *   - upwind DG assembly of one direction on the hex Q1 mesh and on a P1
 *     tetrahedral mesh (Eq. weak_form_transport), block-inverse scaling (Sec. 1.3),
 *     right-hand sides (Eq. sn_transport)
 *   - exact sweep: block forward substitution in topological order (Sec. 1.1);
 *     cycles of the element graph (possible on tetrahedra) as strongly connected
 *     components, each solved as one dense block, unknowns in ascending element order
 *   - AIR setup (Sec. 1.2, Sec. 4.1.1 Eq. soc, Sec. 4.1.2 filtering): strength,
 *     PMIS CF splitting with seeded hashed keys, one-point P, distance-1/2 lAIR
 *     or degree-1 nAIR R = [Z, I], Galerkin R A P
 *   - V-cycle with FC-Jacobi post-relaxation, AIR solve loop
 *   - source iteration with quadrature sum (Eq. angular_quad, Eq. sn_transport)
 *   - adjoint source iteration and cross-section gradients (hex and tetrahedra)
 *
 * Readings where the paper is silent (it defers AIR internals to its refs):
 *   strength uses |a_ij| >= theta * max_{k != i} |a_ik| (empty if the max is 0);
 *   PMIS key = (lambda_i, h_i, i) compared lexicographically, h_i = top 32 bits
 *   of SplitMix64 at state seed ^ (level << 40) ^ i; lambda_i = 0 -> F;
 *   one-point P takes the strongest C neighbour (first maximum);
 *   distance-2 pattern = strong F neighbours of the distance-1 pattern;
 *   nAIR degree 1 = the Neumann series of the strong part of A_FF cut after the
 *   linear term, on the distance-2 pattern (see nair1);
 *   V-cycle: no pre-relaxation; post-relaxation f_sweeps F-Jacobi sweeps then one
 *   C-Jacobi sweep (default 2: the F-F-C ordering usual for AIR); coarsest level
 *   'coarse_sweeps' Jacobi sweeps.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG (-1)
#define OR_ERR_OOM (-2)
#define OR_ERR_SINGULAR (-3)
#define OR_ERR_NOT_CONVERGED (-4)
#define OR_ERR_CYCLE (-9)

#define OR_MAXLEV 64

static const double OR_PI = 3.14159265358979323846;

/* ------------------------------------------------------------------------- */
/* Dense LU with partial pivoting (row-major n x n).                          */
/* Pivot = first row with the largest |entry| in the column; full rows are    */
/* swapped (LAPACK convention P A = L U); multipliers l = a_rk * (1 / a_kk)   */
/* stored below the diagonal; updates a_rc <- fma(-l, a_kc, a_rc) (one        */
/* rounding).  Singular if the pivot magnitude is not above 'tiny'.           */
/* skip_zero: a row whose multiplier is zero gets no update (its update adds   */
/* exact zeros, so only the sign of a zero entry could differ); the lAIR local */
/* systems use it, where most multipliers are zero.                          */
/* ------------------------------------------------------------------------- */
static int lu_factor(int n, double *a, int *piv, double tiny, int skip_zero)
{
    for (int k = 0; k < n; ++k) {
        int p = k;
        double mx = fabs(a[k * n + k]);
        for (int r = k + 1; r < n; ++r) {
            double v = fabs(a[r * n + k]);
            if (v > mx) { mx = v; p = r; }
        }
        piv[k] = p;
        if (!(mx > tiny)) return 1;
        if (p != k) {
            for (int c = 0; c < n; ++c) {
                double t = a[k * n + c]; a[k * n + c] = a[p * n + c]; a[p * n + c] = t;
            }
        }
        double rd = 1.0 / a[k * n + k];
        for (int r = k + 1; r < n; ++r) {
            double l = a[r * n + k] * rd;
            a[r * n + k] = l;
            if (skip_zero && l == 0.0) continue;
            for (int c = k + 1; c < n; ++c) a[r * n + c] = fma(-l, a[k * n + c], a[r * n + c]);
        }
    }
    return 0;
}

/* Transposed solve with the factors of P A = L U: A^T x = y is
 * U^T w = y, L^T v = w, x = P^T v (swaps undone in reverse order). */
static void lu_solve_transpose(int n, const double *a, const int *piv, double *y)
{
    for (int k = 0; k < n; ++k) {
        double s = y[k];
        for (int r = 0; r < k; ++r) s = s - a[r * n + k] * y[r];
        y[k] = s / a[k * n + k];
    }
    for (int k = n - 1; k >= 0; --k) {
        double s = y[k];
        for (int r = k + 1; r < n; ++r) s = s - a[r * n + k] * y[r];
        y[k] = s;
    }
    for (int k = n - 1; k >= 0; --k)
        if (piv[k] != k) { double t = y[k]; y[k] = y[piv[k]]; y[piv[k]] = t; }
}

/* Solve with the factors: swaps in order, unit-lower forward substitution by
 * columns, upper back substitution by columns (y_k <- y_k * (1 / u_kk)). */
static void lu_solve(int n, const double *a, const int *piv, double *y)
{
    for (int k = 0; k < n; ++k)
        if (piv[k] != k) { double t = y[k]; y[k] = y[piv[k]]; y[piv[k]] = t; }
    for (int k = 0; k < n; ++k)
        for (int r = k + 1; r < n; ++r) y[r] = fma(-a[r * n + k], y[k], y[r]);
    for (int k = n - 1; k >= 0; --k) {
        y[k] = y[k] * (1.0 / a[k * n + k]);
        for (int r = 0; r < k; ++r) y[r] = fma(-a[r * n + k], y[k], y[r]);
    }
}

/* ------------------------------------------------------------------------- */
/* DG operator of one direction, element-block form (any element type).      */
/* ------------------------------------------------------------------------- */
typedef struct {
    int E, nb, nfmax, nfn;
    double *D0;     /* E*nb*nb  diagonal block L_KK (unfactored) */
    double *D;      /* E*nb*nb  LU factors of L_KK */
    int *piv;       /* E*nb */
    double *Mass;   /* E*nb*nb  element mass matrix */
    int *nbr;       /* E*nfmax  upwind element across inflow face slot f, -1 if none */
    int *fnodes;    /* E*nfmax*nfn  upwind element's local DOFs on the face, ascending */
    double *Bcol;   /* E*nfmax*nfn*nb  column fnodes[t] of the coupling block L_KK' */
    int *bnd;       /* E*nfmax  1 if slot f is an inflow face on the domain boundary */
    double *Gb;     /* E*nfmax*nb*nb  |Omega.n| int_F phi_b phi_a on boundary inflow faces */
} odg;

static void odg_free(odg *g)
{
    free(g->D0); free(g->D); free(g->piv); free(g->Mass); free(g->nbr);
    free(g->fnodes); free(g->Bcol); free(g->bnd); free(g->Gb);
    memset(g, 0, sizeof(*g));
}

static int odg_alloc(odg *g, int E, int nb, int nfmax, int nfn)
{
    memset(g, 0, sizeof(*g));
    g->E = E; g->nb = nb; g->nfmax = nfmax; g->nfn = nfn;
    size_t bb = (size_t)E * nb * nb;
    g->D0 = calloc(bb, sizeof(double));
    g->D = calloc(bb, sizeof(double));
    g->piv = calloc((size_t)E * nb, sizeof(int));
    g->Mass = calloc(bb, sizeof(double));
    g->nbr = malloc((size_t)E * nfmax * sizeof(int));
    g->fnodes = calloc((size_t)E * nfmax * nfn, sizeof(int));
    g->Bcol = calloc((size_t)E * nfmax * nfn * nb, sizeof(double));
    g->bnd = calloc((size_t)E * nfmax, sizeof(int));
    g->Gb = calloc((size_t)E * nfmax * nb * nb, sizeof(double));
    if (!g->D0 || !g->D || !g->piv || !g->Mass || !g->nbr || !g->fnodes || !g->Bcol || !g->bnd || !g->Gb) {
        odg_free(g);
        return OR_ERR_OOM;
    }
    for (size_t i = 0; i < (size_t)E * nfmax; ++i) g->nbr[i] = -1;
    return OR_OK;
}

/* Factor every diagonal block (Sec. 1.3: the system is scaled by its block
 * diagonal inverse). */
static int odg_factor(odg *g)
{
    int nb = g->nb;
    for (int e = 0; e < g->E; ++e) {
        memcpy(g->D + (size_t)e * nb * nb, g->D0 + (size_t)e * nb * nb, sizeof(double) * nb * nb);
        if (lu_factor(nb, g->D + (size_t)e * nb * nb, g->piv + (size_t)e * nb, 0.0, 0)) return OR_ERR_SINGULAR;
    }
    return OR_OK;
}

/* ---- hex Q1 on the unit cube, n^3 elements, h = 1/n ---------------------- */
/* Element e = ix + n*(iy + n*iz); local node a = ax + 2 ay + 4 az.
 * 1-D factors on [0,h]: m1[i][j] = int phi_i phi_j = (2 or 1) h / 6,
 * g1[i][j] = int phi_j phi_i' = -1/2 (i = 0), +1/2 (i = 1).
 * L_KK[a][b] = sigma_t (phi_b, phi_a)_K - (phi_b, Omega.grad phi_a)_K
 *              + sum_{outflow faces F} (Omega.n) <phi_b, phi_a>_F
 * L_KK'[a][b] = (Omega.n_K) <phi_b^{K'}, phi_a^K>_F on the inflow face F
 * (Eq. weak_form_transport, upwind trace from K'). */
static int hex_build(int n, const double *om, const double *sigma_t, odg *g)
{
    if (n < 1) return OR_ERR_ARG;
    int E = n * n * n;
    int rc = odg_alloc(g, E, 8, 3, 4);
    if (rc) return rc;
    double h = 1.0 / (double)n;
    double m1[2][2], g1[2][2];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) m1[i][j] = ((i == j) ? 2.0 : 1.0) * h / 6.0;
    g1[0][0] = -0.5; g1[0][1] = -0.5; g1[1][0] = 0.5; g1[1][1] = 0.5;
    int out[3], in[3];
    for (int d = 0; d < 3; ++d) { out[d] = om[d] > 0.0 ? 1 : 0; in[d] = 1 - out[d]; }
    const int stride[3] = {1, n, n * n};
    for (int e = 0; e < E; ++e) {
        int idx[3] = {e % n, (e / n) % n, e / (n * n)};
        double st = sigma_t[e];
        double *Dk = g->D0 + (size_t)e * 64;
        double *Mk = g->Mass + (size_t)e * 64;
        for (int a = 0; a < 8; ++a) {
            int ax = a & 1, ay = (a >> 1) & 1, az = (a >> 2) & 1;
            for (int b = 0; b < 8; ++b) {
                int bx = b & 1, by = (b >> 1) & 1, bz = (b >> 2) & 1;
                double mass = (m1[ax][bx] * m1[ay][by]) * m1[az][bz];
                double gx = (g1[ax][bx] * m1[ay][by]) * m1[az][bz];
                double gy = (m1[ax][bx] * g1[ay][by]) * m1[az][bz];
                double gz = (m1[ax][bx] * m1[ay][by]) * g1[az][bz];
                double adv = (om[0] * gx + om[1] * gy) + om[2] * gz;
                double v = st * mass - adv;
                if (om[0] != 0.0 && ax == out[0] && bx == out[0]) v = v + fabs(om[0]) * (m1[ay][by] * m1[az][bz]);
                if (om[1] != 0.0 && ay == out[1] && by == out[1]) v = v + fabs(om[1]) * (m1[ax][bx] * m1[az][bz]);
                if (om[2] != 0.0 && az == out[2] && bz == out[2]) v = v + fabs(om[2]) * (m1[ax][bx] * m1[ay][by]);
                Dk[a * 8 + b] = v;
                Mk[a * 8 + b] = mass;
            }
        }
        for (int d = 0; d < 3; ++d) {
            if (om[d] == 0.0) continue;   /* faces parallel to Omega carry no flux */
            int has_up = (om[d] > 0.0) ? (idx[d] > 0) : (idx[d] < n - 1);
            double w = fabs(om[d]);
            int slot = e * 3 + d;
            if (has_up) {
                int up = (om[d] > 0.0) ? e - stride[d] : e + stride[d];
                g->nbr[slot] = up;
                int t = 0;
                for (int b = 0; b < 8; ++b) {
                    if (((b >> d) & 1) != out[d]) continue;  /* upwind element's nodes on the face */
                    g->fnodes[(size_t)slot * 4 + t] = b;
                    double *col = g->Bcol + ((size_t)slot * 4 + t) * 8;
                    for (int a = 0; a < 8; ++a) {
                        if (((a >> d) & 1) != in[d]) { col[a] = 0.0; continue; }
                        int ax = a & 1, ay = (a >> 1) & 1, az = (a >> 2) & 1;
                        int bx = b & 1, by = (b >> 1) & 1, bz = (b >> 2) & 1;
                        double f = (d == 0) ? m1[ay][by] * m1[az][bz]
                                 : (d == 1) ? m1[ax][bx] * m1[az][bz] : m1[ax][bx] * m1[ay][by];
                        col[a] = -(w * f);
                    }
                    ++t;
                }
            } else {
                g->bnd[slot] = 1;
                double *G = g->Gb + (size_t)slot * 64;
                for (int a = 0; a < 8; ++a) {
                    int ax = a & 1, ay = (a >> 1) & 1, az = (a >> 2) & 1;
                    for (int b = 0; b < 8; ++b) {
                        int bx = b & 1, by = (b >> 1) & 1, bz = (b >> 2) & 1;
                        if (((a >> d) & 1) != in[d] || ((b >> d) & 1) != in[d]) { G[a * 8 + b] = 0.0; continue; }
                        double f = (d == 0) ? m1[ay][by] * m1[az][bz]
                                 : (d == 1) ? m1[ax][bx] * m1[az][bz] : m1[ax][bx] * m1[ay][by];
                        G[a * 8 + b] = w * f;
                    }
                }
            }
        }
    }
    return odg_factor(g);
}

/* ---- tetrahedra, P1 (linear) DG --------------------------------------------- */
/* Local node a = tet vertex a; face f = the triangle without vertex f.
 * Geometry: e_k = x_k - x_0, c23 = e2 x e3, c31 = e3 x e1, c12 = e1 x e2,
 * det = e1 . c23, grad l1 = c23/det, grad l2 = c31/det, grad l3 = c12/det,
 * grad l0 = -((grad l1 + grad l2) + grad l3), |K| = |det| / 6.
 * od_a = Omega . grad l_a.  Mass (|K|/20)(1 + d_ab); advection (phi_b, Omega.grad phi_a)
 * = od_a |K| / 4; face f: (Omega.n)|F| = -(od_f (3 |K|)), face mass (1 + d_ab)/12 of it. */
static void cross3(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot3(const double *a, const double *b) { return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2]; }

static int tet_build(int T, const double *verts, const int *tets, const int *nbrs, const double *om,
                     const double *sigma_t, odg *g)
{
    int rc = odg_alloc(g, T, 4, 4, 3);
    if (rc) return rc;
    for (int t = 0; t < T; ++t) {
        const int *tv = tets + 4 * t;
        double x[4][3], e[3][3], gr[4][3], od[4], c23[3], c31[3], c12[3];
        for (int a = 0; a < 4; ++a)
            for (int k = 0; k < 3; ++k) x[a][k] = verts[3 * tv[a] + k];
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) e[j][k] = x[j + 1][k] - x[0][k];
        cross3(e[1], e[2], c23);
        cross3(e[2], e[0], c31);
        cross3(e[0], e[1], c12);
        double det = dot3(e[0], c23);
        if (det == 0.0) { odg_free(g); return OR_ERR_SINGULAR; }
        for (int k = 0; k < 3; ++k) {
            gr[1][k] = c23[k] / det;
            gr[2][k] = c31[k] / det;
            gr[3][k] = c12[k] / det;
            gr[0][k] = -((gr[1][k] + gr[2][k]) + gr[3][k]);
        }
        double vol = fabs(det) / 6.0;
        for (int a = 0; a < 4; ++a) od[a] = dot3(om, gr[a]);
        double fl[4];
        for (int f = 0; f < 4; ++f) fl[f] = -(od[f] * (3.0 * vol));
        double st = sigma_t[t];
        double *Dk = g->D0 + (size_t)t * 16, *Mk = g->Mass + (size_t)t * 16;
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                double mass = ((a == b) ? 2.0 : 1.0) * vol / 20.0;
                double v = st * mass - od[a] * vol / 4.0;
                for (int f = 0; f < 4; ++f) {
                    if (!(fl[f] > 0.0) || a == f || b == f) continue;   /* outflow faces holding a and b */
                    v = v + fl[f] * ((a == b) ? 2.0 : 1.0) / 12.0;
                }
                Dk[a * 4 + b] = v;
                Mk[a * 4 + b] = mass;
            }
        for (int f = 0; f < 4; ++f) {
            if (!(fl[f] < 0.0)) continue;   /* inflow faces only (Omega.n == 0: no flux) */
            int slot = t * 4 + f, up = nbrs[4 * t + f];
            if (up >= 0) {
                g->nbr[slot] = up;
                const int *uv = tets + 4 * up;
                int u = 0;
                for (int b = 0; b < 4; ++b) {
                    int onface = 0;
                    for (int a = 0; a < 4; ++a) if (a != f && tv[a] == uv[b]) onface = 1;
                    if (!onface) continue;
                    g->fnodes[(size_t)slot * 3 + u] = b;
                    double *col = g->Bcol + ((size_t)slot * 3 + u) * 4;
                    for (int a = 0; a < 4; ++a)
                        col[a] = (a == f) ? 0.0 : fl[f] * ((tv[a] == uv[b]) ? 2.0 : 1.0) / 12.0;
                    ++u;
                }
                if (u != 3) { odg_free(g); return OR_ERR_ARG; }
            } else {
                g->bnd[slot] = 1;
                double *G = g->Gb + (size_t)slot * 16;
                for (int a = 0; a < 4; ++a)
                    for (int b = 0; b < 4; ++b)
                        G[a * 4 + b] = (a == f || b == f) ? 0.0 : -(fl[f] * ((a == b) ? 2.0 : 1.0) / 12.0);
            }
        }
    }
    return odg_factor(g);
}

/* Row entries of the scaled operator A = D^{-1} L for element e, or of L itself.
 * Columns ascending: the element blocks are visited in increasing element
 * index (the upwind neighbours and e itself). */
typedef struct { int col; double val; } oent;

static int cmp_oent(const void *x, const void *y)
{
    int a = ((const oent *)x)->col, b = ((const oent *)y)->col;
    return (a > b) - (a < b);
}

static int odg_row_count(const odg *g, int e)
{
    int c = 0;
    for (int f = 0; f < g->nfmax; ++f) if (g->nbr[e * g->nfmax + f] >= 0) c += g->nfn;
    return c;
}

/* Build CSR of A (scaled = 1: identity diagonal block stored as its diagonal
 * only, couplings D^{-1} L_KK') or of L (scaled = 0: dense diagonal block). */
static int odg_csr(const odg *g, int scaled, int *rowptr, int *col, double *val)
{
    int nb = g->nb, nfn = g->nfn;
    oent *row = malloc(sizeof(oent) * (size_t)(nb + g->nfmax * nfn));
    double *Y = malloc(sizeof(double) * (size_t)g->nfmax * nfn * nb);
    if (!row || !Y) { free(row); free(Y); return OR_ERR_OOM; }
    int p = 0;
    rowptr[0] = 0;
    for (int e = 0; e < g->E; ++e) {
        /* columns of the scaled coupling blocks: y = D_e^{-1} (column of L_KK') */
        for (int f = 0; f < g->nfmax; ++f) {
            if (g->nbr[e * g->nfmax + f] < 0) continue;
            for (int t = 0; t < nfn; ++t) {
                double *y = Y + ((size_t)f * nfn + t) * nb;
                memcpy(y, g->Bcol + (((size_t)e * g->nfmax + f) * nfn + t) * nb, sizeof(double) * nb);
                if (scaled) lu_solve(nb, g->D + (size_t)e * nb * nb, g->piv + (size_t)e * nb, y);
            }
        }
        for (int a = 0; a < nb; ++a) {
            int k = 0;
            if (scaled) {
                row[k].col = e * nb + a; row[k].val = 1.0; ++k;
            } else {
                for (int b = 0; b < nb; ++b) { row[k].col = e * nb + b; row[k].val = g->D0[(size_t)e * nb * nb + a * nb + b]; ++k; }
            }
            for (int f = 0; f < g->nfmax; ++f) {
                int up = g->nbr[e * g->nfmax + f];
                if (up < 0) continue;
                for (int t = 0; t < nfn; ++t) {
                    row[k].col = up * nb + g->fnodes[((size_t)e * g->nfmax + f) * nfn + t];
                    row[k].val = Y[((size_t)f * nfn + t) * nb + a];
                    ++k;
                }
            }
            qsort(row, k, sizeof(oent), cmp_oent);
            for (int i = 0; i < k; ++i) { col[p] = row[i].col; val[p] = row[i].val; ++p; }
            rowptr[e * nb + a + 1] = p;
        }
    }
    free(row); free(Y);
    return OR_OK;
}

/* Right-hand side of Eq. weak_form_transport for one direction:
 *   b_K = M_K s_K + sum_{boundary inflow faces} |Omega.n| <g, phi_a>_F
 * with s the nodal volumetric source (already including the 1/(4 pi)) and g
 * the nodal inflow values; scaled: b_K <- D_K^{-1} b_K. */
static void odg_rhs(const odg *g, const double *src, const double *ginflow, int scaled, double *b)
{
    int nb = g->nb;
    for (int e = 0; e < g->E; ++e) {
        double *be = b + (size_t)e * nb;
        const double *Mk = g->Mass + (size_t)e * nb * nb;
        for (int a = 0; a < nb; ++a) {
            double s = 0.0;
            for (int c = 0; c < nb; ++c) s = s + Mk[a * nb + c] * src[(size_t)e * nb + c];
            be[a] = s;
        }
        if (ginflow) {
            for (int f = 0; f < g->nfmax; ++f) {
                if (!g->bnd[e * g->nfmax + f]) continue;
                const double *G = g->Gb + ((size_t)e * g->nfmax + f) * nb * nb;
                for (int a = 0; a < nb; ++a) {
                    double s = 0.0;
                    for (int c = 0; c < nb; ++c) s = s + G[a * nb + c] * ginflow[(size_t)e * nb + c];
                    be[a] = be[a] + s;
                }
            }
        }
        if (scaled) lu_solve(nb, g->D + (size_t)e * nb * nb, g->piv + (size_t)e * nb, be);
    }
}

/* CSR transpose with ascending columns (counting sort by column). */
static int csr_transpose(int n, const int *rp, const int *ci, const double *v, int **trp, int **tci, double **tv)
{
    int nnz = rp[n];
    int *r = calloc(n + 1, sizeof(int));
    int *c = malloc(sizeof(int) * (size_t)(nnz > 0 ? nnz : 1));
    double *x = malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    int *fill = calloc(n, sizeof(int));
    if (!r || !c || !x || !fill) { free(r); free(c); free(x); free(fill); return OR_ERR_OOM; }
    for (int p = 0; p < nnz; ++p) r[ci[p] + 1]++;
    for (int i = 0; i < n; ++i) r[i + 1] += r[i];
    for (int i = 0; i < n; ++i)
        for (int p = rp[i]; p < rp[i + 1]; ++p) {
            int j = ci[p], q = r[j] + fill[j]++;
            c[q] = i; x[q] = v[p];
        }
    free(fill);
    *trp = r; *tci = c; *tv = x;
    return OR_OK;
}

int or_csr_transpose(int n, const int *rp, const int *ci, const double *v, int *trp, int *tci, double *tv)
{
    int *r, *c; double *x;
    int rc = csr_transpose(n, rp, ci, v, &r, &c, &x);
    if (rc) return rc;
    memcpy(trp, r, sizeof(int) * (size_t)(n + 1));
    memcpy(tci, c, sizeof(int) * (size_t)rp[n]);
    memcpy(tv, x, sizeof(double) * (size_t)rp[n]);
    free(r); free(c); free(x);
    return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Exact sweep (Sec. 1.1): the scaled operator has identity diagonal blocks   */
/* and is block lower triangular in upwind order, so x_K = b_K - sum A_KK' x_K' */
/* visiting elements in topological order (Kahn, smallest index first).      */
/* ------------------------------------------------------------------------- */
/* Exact block solve of the scaled system (identity diagonal blocks) by
 * strongly connected components of the element dependency graph, visited in
 * dependency order (Tarjan: a component is emitted after every component it
 * depends on).  A component of one element is x_K = b_K - sum A_KK' x_K'; a
 * cycle (possible on tetrahedra) is solved as one dense system by LU, its
 * elements in ascending order.
 * order_out (optional): elements in the visiting order.  Returns the number of
 * components with more than one element in *ncyc (optional). */
int or_sweep_scc(int nrows, int nb, const int *rowptr, const int *col, const double *val, const double *b,
                 double *x, int *order_out, int *ncyc)
{
    if (nrows % nb) return OR_ERR_ARG;
    int E = nrows / nb;
    /* adjacency e -> elements it references (its upwind elements) */
    int *cnt = calloc(E + 1, sizeof(int));
    if (!cnt) return OR_ERR_OOM;
    for (int e = 0; e < E; ++e)
        for (int r = e * nb; r < (e + 1) * nb; ++r)
            for (int p = rowptr[r]; p < rowptr[r + 1]; ++p) if (col[p] / nb != e) cnt[e + 1]++;
    for (int e = 0; e < E; ++e) cnt[e + 1] += cnt[e];
    int *adj = malloc(sizeof(int) * (size_t)(cnt[E] > 0 ? cnt[E] : 1));
    int *fill = calloc(E, sizeof(int));
    int *idx = malloc(sizeof(int) * (size_t)E), *low = malloc(sizeof(int) * (size_t)E);
    int *onst = calloc(E, sizeof(int)), *stk = malloc(sizeof(int) * (size_t)E);
    int *cs = malloc(sizeof(int) * (size_t)E), *ci = malloc(sizeof(int) * (size_t)E);
    int *comp = malloc(sizeof(int) * (size_t)E);
    if (!adj || !fill || !idx || !low || !onst || !stk || !cs || !ci || !comp) return OR_ERR_OOM;
    for (int e = 0; e < E; ++e)
        for (int r = e * nb; r < (e + 1) * nb; ++r)
            for (int p = rowptr[r]; p < rowptr[r + 1]; ++p) {
                int u = col[p] / nb;
                if (u != e) adj[cnt[e] + fill[e]++] = u;
            }
    for (int e = 0; e < E; ++e) idx[e] = -1;
    int counter = 0, sp = 0, done = 0, cyc = 0, rc = OR_OK;
    for (int s0 = 0; s0 < E && rc == OR_OK; ++s0) {
        if (idx[s0] >= 0) continue;
        int cd = 0;
        cs[cd] = s0; ci[cd] = cnt[s0]; cd++;
        idx[s0] = low[s0] = counter++; stk[sp++] = s0; onst[s0] = 1;
        while (cd > 0 && rc == OR_OK) {
            int v = cs[cd - 1];
            if (ci[cd - 1] < cnt[v + 1]) {
                int u = adj[ci[cd - 1]++];
                if (idx[u] < 0) {
                    idx[u] = low[u] = counter++; stk[sp++] = u; onst[u] = 1;
                    cs[cd] = u; ci[cd] = cnt[u]; cd++;
                } else if (onst[u] && idx[u] < low[v]) low[v] = idx[u];
                continue;
            }
            --cd;
            if (cd > 0 && low[v] < low[cs[cd - 1]]) low[cs[cd - 1]] = low[v];
            if (low[v] != idx[v]) continue;
            /* pop one component */
            int k = 0;
            for (;;) { int u = stk[--sp]; onst[u] = 0; comp[k++] = u; if (u == v) break; }
            for (int i = 0; i < k; ++i) if (order_out) order_out[done + i] = comp[i];
            done += k;
            if (k == 1) {
                int e = comp[0];
                for (int r = e * nb; r < (e + 1) * nb; ++r) {
                    double sacc = b[r];
                    for (int p = rowptr[r]; p < rowptr[r + 1]; ++p) {
                        int c = col[p];
                        if (c / nb == e) continue;
                        sacc = sacc - val[p] * x[c];
                    }
                    x[r] = sacc;
                }
                continue;
            }
            /* dense solve of the component, unknowns in ascending element order */
            ++cyc;
            for (int i = 1; i < k; ++i)
                for (int j = i; j > 0 && comp[j - 1] > comp[j]; --j) { int t = comp[j]; comp[j] = comp[j - 1]; comp[j - 1] = t; }
            int m = k * nb;
            double *Ad = calloc((size_t)m * m, sizeof(double)), *y = malloc(sizeof(double) * (size_t)m);
            int *pv = malloc(sizeof(int) * (size_t)m), *pos = malloc(sizeof(int) * (size_t)E);
            if (!Ad || !y || !pv || !pos) { rc = OR_ERR_OOM; break; }
            for (int i = 0; i < E; ++i) pos[i] = -1;
            for (int i = 0; i < k; ++i) pos[comp[i]] = i;
            for (int i = 0; i < k; ++i)
                for (int a = 0; a < nb; ++a) {
                    int r = comp[i] * nb + a, rr = i * nb + a;
                    double sacc = b[r];
                    for (int p = rowptr[r]; p < rowptr[r + 1]; ++p) {
                        int c = col[p], pe = pos[c / nb];
                        if (pe >= 0) Ad[(size_t)rr * m + pe * nb + c % nb] = val[p];
                        else sacc = sacc - val[p] * x[c];
                    }
                    y[rr] = sacc;
                }
            if (lu_factor(m, Ad, pv, 0.0, 0)) rc = OR_ERR_SINGULAR;
            else {
                lu_solve(m, Ad, pv, y);
                for (int i = 0; i < k; ++i)
                    for (int a = 0; a < nb; ++a) x[comp[i] * nb + a] = y[i * nb + a];
            }
            free(Ad); free(y); free(pv); free(pos);
        }
    }
    free(cnt); free(adj); free(fill); free(idx); free(low); free(onst); free(stk); free(cs); free(ci); free(comp);
    if (ncyc) *ncyc = cyc;
    return rc;
}

int or_sweep(int nrows, int nb, const int *rowptr, const int *col, const double *val,
             const double *b, double *x, int *order_out)
{
    return or_sweep_scc(nrows, nb, rowptr, col, val, b, x, order_out, NULL);
}

/* ------------------------------------------------------------------------- */
/* Exported assembly entry points (hex).                                      */
/* ------------------------------------------------------------------------- */
int or_hex_nnz(int n, const double *om, int scaled)
{
    odg g;
    double *st = malloc(sizeof(double) * (size_t)n * n * n);
    if (!st) return OR_ERR_OOM;
    for (int i = 0; i < n * n * n; ++i) st[i] = 1.0;
    int rc = hex_build(n, om, st, &g);
    free(st);
    if (rc) return rc;
    int nnz = 0;
    for (int e = 0; e < g.E; ++e) nnz += g.nb * ((scaled ? 1 : g.nb) + odg_row_count(&g, e));
    odg_free(&g);
    return nnz;
}

int or_hex_assemble(int n, const double *om, const double *sigma_t, int scaled,
                    int *rowptr, int *col, double *val)
{
    odg g;
    int rc = hex_build(n, om, sigma_t, &g);
    if (rc) return rc;
    rc = odg_csr(&g, scaled, rowptr, col, val);
    odg_free(&g);
    return rc;
}

/* src: nodal source values (N), g: nodal inflow values (N) or NULL. */
int or_hex_rhs(int n, const double *om, const double *sigma_t, const double *src,
               const double *ginflow, int scaled, double *b)
{
    odg g;
    int rc = hex_build(n, om, sigma_t, &g);
    if (rc) return rc;
    odg_rhs(&g, src, ginflow, scaled, b);
    odg_free(&g);
    return OR_OK;
}

int or_tet_nnz(int T, const double *verts, const int *tets, const int *nbrs, const double *om, int scaled)
{
    odg g;
    double *st = malloc(sizeof(double) * (size_t)T);
    if (!st) return OR_ERR_OOM;
    for (int i = 0; i < T; ++i) st[i] = 1.0;
    int rc = tet_build(T, verts, tets, nbrs, om, st, &g);
    free(st);
    if (rc) return rc;
    int nnz = 0;
    for (int e = 0; e < T; ++e) nnz += 4 * ((scaled ? 1 : 4) + odg_row_count(&g, e));
    odg_free(&g);
    return nnz;
}

int or_tet_assemble(int T, const double *verts, const int *tets, const int *nbrs, const double *om,
                    const double *sigma_t, int scaled, int *rowptr, int *col, double *val)
{
    odg g;
    int rc = tet_build(T, verts, tets, nbrs, om, sigma_t, &g);
    if (rc) return rc;
    rc = odg_csr(&g, scaled, rowptr, col, val);
    odg_free(&g);
    return rc;
}

int or_tet_rhs(int T, const double *verts, const int *tets, const int *nbrs, const double *om, const double *sigma_t,
               const double *src, const double *ginflow, int scaled, double *b)
{
    odg g;
    int rc = tet_build(T, verts, tets, nbrs, om, sigma_t, &g);
    if (rc) return rc;
    odg_rhs(&g, src, ginflow, scaled, b);
    odg_free(&g);
    return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* AIR setup                                                                  */
/* ------------------------------------------------------------------------- */
typedef struct {
    int distance;
    double theta, eps_R, phi_R, phi_A;
    int max_levels, max_coarse, coarse_sweeps;
    uint64_t seed;
    int f_sweeps;   /* F-Jacobi sweeps before the C-Jacobi sweep (1: FC, 2: FFC) */
    int nair;       /* 0: lAIR; 1: nAIR of degree 1 (Neumann series) */
} or_params;

typedef struct {
    int n, nnz;
    int *rowptr, *col;
    double *val;
    double *dinv;
    int coarsest;
    signed char *cf;   /* 1 C, 0 F (non-coarsest levels) */
    int *pmap;         /* P column per fine row (coarse index) or -1 */
    int nc;
    int *cpts;         /* fine index of every coarse point */
    int *zrowptr, *zcol, nnzZ;
    double *zval;
    int pmis_rounds, n_singular;
} olevel;

typedef struct {
    int nlev;
    or_params prm;
    olevel lev[OR_MAXLEV];
} ohier;

static uint64_t splitmix_first(uint64_t state)
{
    uint64_t z = state + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Strength (Eq. soc, absolute values): j in S_i iff j != i and
 * |a_ij| >= thr * max_{k != i} |a_ik|; empty when that max is zero. */
static void strength(const olevel *L, double thr, signed char *S)
{
    for (int i = 0; i < L->n; ++i) {
        double m = 0.0;
        for (int p = L->rowptr[i]; p < L->rowptr[i + 1]; ++p)
            if (L->col[p] != i) { double v = fabs(L->val[p]); if (v > m) m = v; }
        double t = thr * m;
        for (int p = L->rowptr[i]; p < L->rowptr[i + 1]; ++p)
            S[p] = (L->col[p] != i && m > 0.0 && fabs(L->val[p]) >= t) ? 1 : 0;
    }
}

typedef struct { uint32_t lam, h; int i; } okey;
static int key_gt(okey a, okey b)
{
    if (a.lam != b.lam) return a.lam > b.lam;
    if (a.h != b.h) return a.h > b.h;
    return a.i > b.i;
}

/* PMIS (De Sterck, Yang, Heys) with a deterministic key.  cf: 1 C, 0 F. */
static int pmis(const olevel *L, const signed char *S, int level, uint64_t seed, signed char *cf, int *rounds)
{
    int n = L->n;
    enum { U = -1 };
    uint32_t *lam = calloc(n, sizeof(uint32_t));
    int *tp = calloc(n + 1, sizeof(int));
    if (!lam || !tp) { free(lam); free(tp); return OR_ERR_OOM; }
    for (int i = 0; i < n; ++i)
        for (int p = L->rowptr[i]; p < L->rowptr[i + 1]; ++p)
            if (S[p]) { lam[L->col[p]]++; tp[L->col[p] + 1]++; }
    for (int i = 0; i < n; ++i) tp[i + 1] += tp[i];
    int *st = malloc(sizeof(int) * (size_t)(tp[n] > 0 ? tp[n] : 1));   /* S^T lists */
    int *fill = calloc(n, sizeof(int));
    okey *key = malloc(sizeof(okey) * (size_t)(n > 0 ? n : 1));
    signed char *newc = calloc(n, 1);
    if (!st || !fill || !key || !newc) { free(lam); free(tp); free(st); free(fill); free(key); free(newc); return OR_ERR_OOM; }
    for (int i = 0; i < n; ++i)
        for (int p = L->rowptr[i]; p < L->rowptr[i + 1]; ++p)
            if (S[p]) { int j = L->col[p]; st[tp[j] + fill[j]++] = i; }
    for (int i = 0; i < n; ++i) {
        key[i].lam = lam[i];
        key[i].h = (uint32_t)(splitmix_first(seed ^ ((uint64_t)level << 40) ^ (uint64_t)i) >> 32);
        key[i].i = i;
        cf[i] = lam[i] == 0 ? 0 : U;
    }
    int r = 0;
    for (;;) {
        int undecided = 0;
        for (int i = 0; i < n; ++i) undecided += (cf[i] == U);
        if (!undecided) break;
        ++r;
        for (int i = 0; i < n; ++i) {
            newc[i] = 0;
            if (cf[i] != U) continue;
            int ismax = 1;
            for (int p = L->rowptr[i]; p < L->rowptr[i + 1] && ismax; ++p)
                if (S[p] && cf[L->col[p]] == U && key_gt(key[L->col[p]], key[i])) ismax = 0;
            for (int k = tp[i]; k < tp[i + 1] && ismax; ++k)
                if (cf[st[k]] == U && key_gt(key[st[k]], key[i])) ismax = 0;
            newc[i] = (signed char)ismax;
        }
        for (int i = 0; i < n; ++i) if (newc[i]) cf[i] = 1;
        for (int i = 0; i < n; ++i) {
            if (cf[i] != U) continue;
            for (int p = L->rowptr[i]; p < L->rowptr[i + 1]; ++p)
                if (S[p] && cf[L->col[p]] == 1) { cf[i] = 0; break; }
        }
    }
    *rounds = r;
    free(lam); free(tp); free(st); free(fill); free(key); free(newc);
    return OR_OK;
}

static double lookup(const olevel *L, int i, int j)
{
    int lo = L->rowptr[i], hi = L->rowptr[i + 1] - 1;
    while (lo <= hi) {
        int m = (lo + hi) / 2;
        if (L->col[m] == j) return L->val[m];
        if (L->col[m] < j) lo = m + 1; else hi = m - 1;
    }
    return 0.0;
}

static int cmp_int(const void *x, const void *y)
{
    int a = *(const int *)x, b = *(const int *)y;
    return (a > b) - (a < b);
}

/* lAIR (Sec. 1.2; Sec. 4.1.1): for every C point i, with pattern Rp of strong
 * F neighbours (distance 1, or 2 through F points), solve
 *   A[Rp,Rp]^T z = -A[i,Rp]^T
 * so that (Z A_FF + A_CF)[i, Rp] = 0; then the optional filter of Sec. 4.1.2
 * drops |z_j| < phi_R max_k |z_k|. */
static int lair(olevel *L, const signed char *SR, int distance, double phi_R)
{
    int n = L->n, nc = L->nc;
    L->zrowptr = calloc(nc + 1, sizeof(int));
    int cap = 1024, used = 0;
    L->zcol = malloc(sizeof(int) * cap);
    L->zval = malloc(sizeof(double) * cap);
    int *pat = malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int *mark = malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    if (!L->zrowptr || !L->zcol || !L->zval || !pat || !mark) { free(pat); free(mark); return OR_ERR_OOM; }
    for (int i = 0; i < n; ++i) mark[i] = -1;
    L->n_singular = 0;
    for (int ic = 0; ic < nc; ++ic) {
        int i = L->cpts[ic];
        int np = 0;
        for (int p = L->rowptr[i]; p < L->rowptr[i + 1]; ++p) {
            int j = L->col[p];
            if (SR[p] && L->cf[j] == 0 && mark[j] != ic) { mark[j] = ic; pat[np++] = j; }
        }
        if (distance >= 2) {
            int n1 = np;
            for (int t = 0; t < n1; ++t) {
                int j = pat[t];
                for (int p = L->rowptr[j]; p < L->rowptr[j + 1]; ++p) {
                    int k = L->col[p];
                    if (SR[p] && L->cf[k] == 0 && mark[k] != ic) { mark[k] = ic; pat[np++] = k; }
                }
            }
        }
        qsort(pat, np, sizeof(int), cmp_int);
        double *M = malloc(sizeof(double) * (size_t)(np > 0 ? np * np : 1));
        double *z = malloc(sizeof(double) * (size_t)(np > 0 ? np : 1));
        int *piv = malloc(sizeof(int) * (size_t)(np > 0 ? np : 1));
        if (!M || !z || !piv) { free(M); free(z); free(piv); free(pat); free(mark); return OR_ERR_OOM; }
        double mx = 0.0;
        for (int r = 0; r < np; ++r) {
            for (int c = 0; c < np; ++c) {
                double v = lookup(L, pat[c], pat[r]);   /* transpose */
                M[r * np + c] = v;
                if (fabs(v) > mx) mx = fabs(v);
            }
            z[r] = -lookup(L, i, pat[r]);
        }
        int keep = np;
        if (np > 0) {
            if (lu_factor(np, M, piv, 1e-14 * mx, 1)) { L->n_singular++; keep = 0; }
            else lu_solve(np, M, piv, z);
        }
        double zmax = 0.0;
        for (int t = 0; t < keep; ++t) if (fabs(z[t]) > zmax) zmax = fabs(z[t]);
        double thr = phi_R * zmax;
        for (int t = 0; t < keep; ++t) {
            if (phi_R > 0.0 && fabs(z[t]) < thr) continue;
            if (used == cap) {
                cap *= 2;
                L->zcol = realloc(L->zcol, sizeof(int) * cap);
                L->zval = realloc(L->zval, sizeof(double) * cap);
                if (!L->zcol || !L->zval) { free(M); free(z); free(piv); free(pat); free(mark); return OR_ERR_OOM; }
            }
            L->zcol[used] = pat[t]; L->zval[used] = z[t]; ++used;
        }
        L->zrowptr[ic + 1] = used;
        free(M); free(z); free(piv);
    }
    L->nnzZ = used;
    free(pat); free(mark);
    return OR_OK;
}

/* nAIR of degree 1 (Sec. 1.2: the Neumann-expansion variant of AIR; the
 * best-scaling runs of Sec. 4.1.2 use it with phi_R = 0.1).  With only the strong
 * (eps_R) entries of A_FF and A_CF kept (marked s), D the diagonal of A_FF and
 * N = I - D^{-1} A_FF^s, so that A_FF^s = D (I - N), the ideal restriction
 * -A_CF^s (A_FF^s)^{-1} = -A_CF^s (I + N + N^2 + ...) D^{-1} is cut after the
 * linear term:
 *   Z_i = -A_CF^s[i, :] (I + N) D^{-1}
 * on the strong F neighbours of i and their strong F neighbours.  Entry k:
 *   t_k = a_ik (k a strong F neighbour of i, else 0), then for every strong F
 *   neighbour j of i in ascending order and every strong F neighbour k != j of j,
 *   t_k = fma(a_ij, n_jk, t_k) with n_jk = -(a_jk * (1/a_jj));
 *   z_k = -(t_k * (1/a_kk)).
 * A zero diagonal on the way makes the row empty (counted as singular).  Then the
 * filter of Sec. 4.1.2 as in lAIR. */
static int nair1(olevel *L, const signed char *SR, double phi_R)
{
    int n = L->n, nc = L->nc;
    L->zrowptr = calloc(nc + 1, sizeof(int));
    int cap = 1024, used = 0;
    L->zcol = malloc(sizeof(int) * cap);
    L->zval = malloc(sizeof(double) * cap);
    int *pat = malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int *mark = malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int *pos = malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    double *t = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!L->zrowptr || !L->zcol || !L->zval || !pat || !mark || !pos || !t) {
        free(pat); free(mark); free(pos); free(t); return OR_ERR_OOM;
    }
    for (int i = 0; i < n; ++i) mark[i] = -1;
    L->n_singular = 0;
    for (int ic = 0; ic < nc; ++ic) {
        int i = L->cpts[ic];
        int np = 0;
        for (int p = L->rowptr[i]; p < L->rowptr[i + 1]; ++p) {
            int j = L->col[p];
            if (SR[p] && L->cf[j] == 0 && mark[j] != ic) { mark[j] = ic; pat[np++] = j; }
        }
        int n1 = np;
        for (int a = 0; a < n1; ++a) {
            int j = pat[a];
            for (int p = L->rowptr[j]; p < L->rowptr[j + 1]; ++p) {
                int k = L->col[p];
                if (SR[p] && L->cf[k] == 0 && mark[k] != ic) { mark[k] = ic; pat[np++] = k; }
            }
        }
        qsort(pat, np, sizeof(int), cmp_int);
        for (int a = 0; a < np; ++a) { pos[pat[a]] = a; t[a] = 0.0; }
        int singular = 0;
        for (int p = L->rowptr[i]; p < L->rowptr[i + 1]; ++p) {
            int k = L->col[p];
            if (SR[p] && L->cf[k] == 0) t[pos[k]] = L->val[p];
        }
        for (int p = L->rowptr[i]; p < L->rowptr[i + 1] && !singular; ++p) {
            int j = L->col[p];
            if (!(SR[p] && L->cf[j] == 0)) continue;
            double aij = L->val[p], rj = L->dinv[j];
            if (rj == 0.0) { singular = 1; break; }
            for (int q = L->rowptr[j]; q < L->rowptr[j + 1]; ++q) {
                int k = L->col[q];
                if (k == j || !(SR[q] && L->cf[k] == 0)) continue;
                double njk = -(L->val[q] * rj);
                t[pos[k]] = fma(aij, njk, t[pos[k]]);
            }
        }
        for (int a = 0; a < np && !singular; ++a)
            if (L->dinv[pat[a]] == 0.0) singular = 1;
        int keep = np;
        if (singular) { L->n_singular++; keep = 0; }
        for (int a = 0; a < keep; ++a) t[a] = -(t[a] * L->dinv[pat[a]]);
        double zmax = 0.0;
        for (int a = 0; a < keep; ++a) if (fabs(t[a]) > zmax) zmax = fabs(t[a]);
        double thr = phi_R * zmax;
        for (int a = 0; a < keep; ++a) {
            if (phi_R > 0.0 && fabs(t[a]) < thr) continue;
            if (used == cap) {
                cap *= 2;
                L->zcol = realloc(L->zcol, sizeof(int) * cap);
                L->zval = realloc(L->zval, sizeof(double) * cap);
                if (!L->zcol || !L->zval) { free(pat); free(mark); free(pos); free(t); return OR_ERR_OOM; }
            }
            L->zcol[used] = pat[a]; L->zval[used] = t[a]; ++used;
        }
        L->zrowptr[ic + 1] = used;
    }
    L->nnzZ = used;
    free(pat); free(mark); free(pos); free(t);
    return OR_OK;
}

/* Galerkin coarse operator A_c = R A P (Sec. 1.2; Sec. 4.1.2 stencil growth).
 * (AP)[k,c] = sum_l a_kl over l ascending with pmap(l) = c;
 * (RAP)[ic,c] = sum_k R[ic,k] (AP)[k,c] over the R row in ascending column
 * order, the identity entry (k = C point of ic) included in place, each term
 * accumulated with one fused multiply-add.
 * Every structural product is kept (exact zeros included). */
static int rap(const olevel *L, olevel *C, double phi_A)
{
    int n = L->n, nc = L->nc;
    /* AP rows */
    int *aprow = malloc(sizeof(int) * (size_t)(n + 1));
    int *apcol = malloc(sizeof(int) * (size_t)(L->nnz > 0 ? L->nnz : 1));
    double *apval = malloc(sizeof(double) * (size_t)(L->nnz > 0 ? L->nnz : 1));
    double *acc = malloc(sizeof(double) * (size_t)(nc > 0 ? nc : 1));
    int *where = malloc(sizeof(int) * (size_t)(nc > 0 ? nc : 1));
    int *list = malloc(sizeof(int) * (size_t)(nc > 0 ? nc : 1));
    if (!aprow || !apcol || !apval || !acc || !where || !list) return OR_ERR_OOM;
    for (int c = 0; c < nc; ++c) where[c] = -1;
    int q = 0;
    aprow[0] = 0;
    for (int k = 0; k < n; ++k) {
        int nl = 0;
        for (int p = L->rowptr[k]; p < L->rowptr[k + 1]; ++p) {
            int c = L->pmap[L->col[p]];
            if (c < 0) continue;
            if (where[c] < 0) { where[c] = nl; list[nl++] = c; acc[c] = 0.0; }
            acc[c] = acc[c] + L->val[p];
        }
        qsort(list, nl, sizeof(int), cmp_int);
        for (int t = 0; t < nl; ++t) { apcol[q] = list[t]; apval[q] = acc[list[t]]; where[list[t]] = -1; ++q; }
        aprow[k + 1] = q;
    }
    /* RAP rows */
    int cap = 1024, used = 0;
    int *ccol = malloc(sizeof(int) * cap);
    double *cval = malloc(sizeof(double) * cap);
    int *crow = malloc(sizeof(int) * (size_t)(nc + 1));
    int *rc_ = malloc(sizeof(int) * (size_t)(L->nnzZ + nc > 0 ? L->nnzZ + nc : 1));
    double *rv_ = malloc(sizeof(double) * (size_t)(L->nnzZ + nc > 0 ? L->nnzZ + nc : 1));
    if (!ccol || !cval || !crow || !rc_ || !rv_) return OR_ERR_OOM;
    crow[0] = 0;
    for (int ic = 0; ic < nc; ++ic) {
        /* R row: Z entries plus the identity at the C point, ascending */
        int i = L->cpts[ic], nr = 0, placed = 0;
        for (int t = L->zrowptr[ic]; t < L->zrowptr[ic + 1]; ++t) {
            if (!placed && L->zcol[t] > i) { rc_[nr] = i; rv_[nr] = 1.0; ++nr; placed = 1; }
            rc_[nr] = L->zcol[t]; rv_[nr] = L->zval[t]; ++nr;
        }
        if (!placed) { rc_[nr] = i; rv_[nr] = 1.0; ++nr; }
        int nl = 0;
        for (int t = 0; t < nr; ++t) {
            int k = rc_[t];
            double r = rv_[t];
            for (int p = aprow[k]; p < aprow[k + 1]; ++p) {
                int c = apcol[p];
                if (where[c] < 0) { where[c] = nl; list[nl++] = c; acc[c] = 0.0; }
                acc[c] = fma(r, apval[p], acc[c]);
            }
        }
        qsort(list, nl, sizeof(int), cmp_int);
        /* optional coarse filter: drop |a_ij| < phi_A max_{j != i} |a_ij|, keep the diagonal */
        double mx = 0.0;
        for (int t = 0; t < nl; ++t) if (list[t] != ic && fabs(acc[list[t]]) > mx) mx = fabs(acc[list[t]]);
        double thr = phi_A * mx;
        for (int t = 0; t < nl; ++t) {
            int c = list[t];
            where[c] = -1;
            if (phi_A > 0.0 && c != ic && fabs(acc[c]) < thr) continue;
            if (used == cap) {
                cap *= 2;
                ccol = realloc(ccol, sizeof(int) * cap);
                cval = realloc(cval, sizeof(double) * cap);
                if (!ccol || !cval) return OR_ERR_OOM;
            }
            ccol[used] = c; cval[used] = acc[c]; ++used;
        }
        crow[ic + 1] = used;
    }
    C->n = nc; C->nnz = used; C->rowptr = crow; C->col = ccol; C->val = cval;
    free(aprow); free(apcol); free(apval); free(acc); free(where); free(list); free(rc_); free(rv_);
    return OR_OK;
}

static void level_dinv(olevel *L)
{
    L->dinv = malloc(sizeof(double) * (size_t)(L->n > 0 ? L->n : 1));
    for (int i = 0; i < L->n; ++i) {
        double d = lookup(L, i, i);
        L->dinv[i] = (d != 0.0) ? 1.0 / d : 0.0;
    }
}

static void level_free(olevel *L)
{
    free(L->rowptr); free(L->col); free(L->val); free(L->dinv); free(L->cf); free(L->pmap);
    free(L->cpts); free(L->zrowptr); free(L->zcol); free(L->zval);
    memset(L, 0, sizeof(*L));
}

void or_hier_free(void *hp)
{
    ohier *H = hp;
    if (!H) return;
    for (int l = 0; l < H->nlev; ++l) level_free(&H->lev[l]);
    free(H);
}

void or_params_default(or_params *p)
{
    p->distance = 1; p->theta = 0.25; p->eps_R = 0.01; p->phi_R = 0.0; p->phi_A = 0.0;
    p->max_levels = 25; p->max_coarse = 100; p->coarse_sweeps = 20; p->seed = 3; p->f_sweeps = 2;
    p->nair = 0;
}

/* AIR setup on a CSR matrix with sorted columns (copied). */
void *or_air_setup(int n, const int *rowptr, const int *col, const double *val, const or_params *prm, int *status)
{
    ohier *H = calloc(1, sizeof(ohier));
    if (!H) { *status = OR_ERR_OOM; return NULL; }
    H->prm = *prm;
    olevel *L0 = &H->lev[0];
    L0->n = n; L0->nnz = rowptr[n];
    L0->rowptr = malloc(sizeof(int) * (size_t)(n + 1));
    L0->col = malloc(sizeof(int) * (size_t)(L0->nnz > 0 ? L0->nnz : 1));
    L0->val = malloc(sizeof(double) * (size_t)(L0->nnz > 0 ? L0->nnz : 1));
    memcpy(L0->rowptr, rowptr, sizeof(int) * (size_t)(n + 1));
    memcpy(L0->col, col, sizeof(int) * (size_t)L0->nnz);
    memcpy(L0->val, val, sizeof(double) * (size_t)L0->nnz);
    H->nlev = 1;
    *status = OR_OK;
    for (int l = 0;; ++l) {
        olevel *L = &H->lev[l];
        level_dinv(L);
        if (L->n <= prm->max_coarse || l == prm->max_levels - 1 || l == OR_MAXLEV - 1) { L->coarsest = 1; break; }
        signed char *S = malloc((size_t)(L->nnz > 0 ? L->nnz : 1));
        signed char *SR = malloc((size_t)(L->nnz > 0 ? L->nnz : 1));
        L->cf = malloc((size_t)(L->n > 0 ? L->n : 1));
        strength(L, prm->theta, S);
        strength(L, prm->eps_R, SR);
        int rc = pmis(L, S, l, prm->seed, L->cf, &L->pmis_rounds);
        if (rc) { *status = rc; free(S); free(SR); break; }
        int nc = 0;
        for (int i = 0; i < L->n; ++i) nc += (L->cf[i] == 1);
        if (nc == 0 || (double)nc >= 0.9 * (double)L->n) {
            L->coarsest = 1; free(L->cf); L->cf = NULL; free(S); free(SR); break;
        }
        L->nc = nc;
        L->cpts = malloc(sizeof(int) * (size_t)nc);
        L->pmap = malloc(sizeof(int) * (size_t)L->n);
        int *cmap = malloc(sizeof(int) * (size_t)L->n);
        for (int i = 0, c = 0; i < L->n; ++i) { cmap[i] = -1; if (L->cf[i] == 1) { cmap[i] = c; L->cpts[c++] = i; } }
        /* one-point interpolation (Sec. 1.2: C points interpolated by value):
         * F row -> strongest C neighbour in S_i (first maximum), else empty */
        for (int i = 0; i < L->n; ++i) {
            if (L->cf[i] == 1) { L->pmap[i] = cmap[i]; continue; }
            int best = -1; double bv = -1.0;
            for (int p = L->rowptr[i]; p < L->rowptr[i + 1]; ++p) {
                int j = L->col[p];
                if (S[p] && L->cf[j] == 1 && fabs(L->val[p]) > bv) { bv = fabs(L->val[p]); best = j; }
            }
            L->pmap[i] = best >= 0 ? cmap[best] : -1;
        }
        free(cmap);
        rc = prm->nair ? nair1(L, SR, prm->phi_R) : lair(L, SR, prm->distance, prm->phi_R);
        free(S); free(SR);
        if (rc) { *status = rc; break; }
        rc = rap(L, &H->lev[l + 1], prm->phi_A);
        if (rc) { *status = rc; break; }
        H->nlev = l + 2;
    }
    return H;
}

int or_hier_nlev(void *hp) { return ((ohier *)hp)->nlev; }

/* sizes: n, nnz, nc, nnzZ, coarsest, pmis_rounds, n_singular */
void or_hier_level_sizes(void *hp, int l, int *out)
{
    olevel *L = &((ohier *)hp)->lev[l];
    out[0] = L->n; out[1] = L->nnz; out[2] = L->nc; out[3] = L->nnzZ;
    out[4] = L->coarsest; out[5] = L->pmis_rounds; out[6] = L->n_singular;
}

void or_hier_level_export(void *hp, int l, int *rowptr, int *col, double *val, double *dinv,
                          signed char *cf, int *pmap, int *cpts, int *zrowptr, int *zcol, double *zval)
{
    olevel *L = &((ohier *)hp)->lev[l];
    if (rowptr) memcpy(rowptr, L->rowptr, sizeof(int) * (size_t)(L->n + 1));
    if (col) memcpy(col, L->col, sizeof(int) * (size_t)L->nnz);
    if (val) memcpy(val, L->val, sizeof(double) * (size_t)L->nnz);
    if (dinv) memcpy(dinv, L->dinv, sizeof(double) * (size_t)L->n);
    if (L->coarsest) return;
    if (cf) memcpy(cf, L->cf, (size_t)L->n);
    if (pmap) memcpy(pmap, L->pmap, sizeof(int) * (size_t)L->n);
    if (cpts) memcpy(cpts, L->cpts, sizeof(int) * (size_t)L->nc);
    if (zrowptr) memcpy(zrowptr, L->zrowptr, sizeof(int) * (size_t)(L->nc + 1));
    if (zcol) memcpy(zcol, L->zcol, sizeof(int) * (size_t)L->nnzZ);
    if (zval) memcpy(zval, L->zval, sizeof(double) * (size_t)L->nnzZ);
}

/* ------------------------------------------------------------------------- */
/* V-cycle and solve                                                          */
/* ------------------------------------------------------------------------- */
static void residual(const olevel *L, const double *b, const double *x, double *r)
{
    for (int i = 0; i < L->n; ++i) {
        double s = 0.0;
        for (int p = L->rowptr[i]; p < L->rowptr[i + 1]; ++p) s = s + L->val[p] * x[L->col[p]];
        r[i] = b[i] - s;
    }
}

static void vcycle_level(const ohier *H, int l, const double *b, double *x)
{
    const olevel *L = &H->lev[l];
    int n = L->n;
    double *r = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (L->coarsest) {
        /* coarsest level: pointwise Jacobi sweeps */
        for (int s = 0; s < H->prm.coarse_sweeps; ++s) {
            residual(L, b, x, r);
            for (int i = 0; i < n; ++i) x[i] = x[i] + L->dinv[i] * r[i];
        }
        free(r);
        return;
    }
    int nc = L->nc;
    residual(L, b, x, r);
    /* restriction: bc = R r, R row = [Z_i, 1] in ascending column order */
    double *bc = malloc(sizeof(double) * (size_t)nc);
    double *xc = calloc(nc, sizeof(double));
    for (int ic = 0; ic < nc; ++ic) {
        int i = L->cpts[ic], placed = 0;
        double s = 0.0;
        for (int t = L->zrowptr[ic]; t < L->zrowptr[ic + 1]; ++t) {
            if (!placed && L->zcol[t] > i) { s = s + r[i]; placed = 1; }
            s = s + L->zval[t] * r[L->zcol[t]];
        }
        if (!placed) s = s + r[i];
        bc[ic] = s;
    }
    vcycle_level(H, l + 1, bc, xc);
    /* one-point prolongation: x_i += xc[pmap(i)] */
    for (int i = 0; i < n; ++i) if (L->pmap[i] >= 0) x[i] = x[i] + xc[L->pmap[i]];
    /* post-relaxation: f_sweeps F-Jacobi sweeps, then C-Jacobi (omega = 1) */
    for (int s = 0; s < H->prm.f_sweeps; ++s) {
        residual(L, b, x, r);
        for (int i = 0; i < n; ++i) if (L->cf[i] == 0) x[i] = x[i] + L->dinv[i] * r[i];
    }
    residual(L, b, x, r);
    for (int i = 0; i < n; ++i) if (L->cf[i] == 1) x[i] = x[i] + L->dinv[i] * r[i];
    free(r); free(bc); free(xc);
}

void or_vcycle(void *hp, const double *b, double *x) { vcycle_level(hp, 0, b, x); }

static double norm2(int n, const double *v)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i) s = s + v[i] * v[i];
    return sqrt(s);
}

/* AIR iterations until ||b - A x|| <= tol ||b|| (Sec. 2.1).  hist[k] holds the
 * residual norm after k cycles (k = 0..iters). */
int or_air_solve(void *hp, const double *b, double *x, double tol, int maxit, int *iters, double *hist)
{
    ohier *H = hp;
    const olevel *L = &H->lev[0];
    double *r = malloc(sizeof(double) * (size_t)(L->n > 0 ? L->n : 1));
    double bn = norm2(L->n, b);
    residual(L, b, x, r);
    double rn = norm2(L->n, r);
    if (hist) hist[0] = rn;
    int k = 0;
    while (rn > tol * bn && k < maxit) {
        vcycle_level(H, 0, b, x);
        residual(L, b, x, r);
        rn = norm2(L->n, r);
        ++k;
        if (hist) hist[k] = rn;
    }
    free(r);
    *iters = k;
    return rn <= tol * bn ? OR_OK : OR_ERR_NOT_CONVERGED;
}

/* ------------------------------------------------------------------------- */
/* Source iteration (Eq. sn_transport) on the hex mesh                        */
/* ------------------------------------------------------------------------- */
typedef struct {
    double tol;         /* ||phi^{n+1} - phi^n|| / ||phi^{n+1}|| */
    int max_iters;
    double inner_tol;   /* relative residual of each direction's solve */
    int inner_maxit;
    int use_sweep;      /* 1: exact sweep instead of AIR */
    double g_inflow;    /* isotropic inflow angular flux on the inflow boundary */
    int inner_cycles;   /* > 0: every direction's solve is exactly this many V-cycles from
                           zero, a fixed approximate inverse (Sec. 3: source iteration then
                           converges to the modified problem with that inverse) */
    const double *q_ang; /* NULL, or M*N nodal values of an angular source density added to
                            direction m's right-hand side (direction-major), e.g. a
                            manufactured-solution source (Appendix) */
} or_si_params;

/* Mesh descriptor: kind 0 = n^3 hexahedra (Q1), kind 1 = tetrahedra (P1). */
typedef struct {
    int kind, n, T;
    const double *verts;
    const int *tets, *nbr;
} or_mesh;

static int mesh_build(const or_mesh *mesh, const double *om, const double *sigma_t, odg *g)
{
    if (mesh->kind == 0) return hex_build(mesh->n, om, sigma_t, g);
    if (mesh->kind == 1) return tet_build(mesh->T, mesh->verts, mesh->tets, mesh->nbr, om, sigma_t, g);
    return OR_ERR_ARG;
}

typedef struct {
    odg g;
    int nnz;
    int *rowptr, *col;
    double *val;
    void *hier;
} odir;

static void odir_free(odir *d)
{
    odg_free(&d->g); free(d->rowptr); free(d->col); free(d->val);
    if (d->hier) or_hier_free(d->hier);
}

static int odir_build(odir *d, const or_mesh *mesh, const double *om, const double *sigma_t, const or_params *prm,
                      int with_air)
{
    memset(d, 0, sizeof(*d));
    int rc = mesh_build(mesh, om, sigma_t, &d->g);
    if (rc) return rc;
    int N = d->g.E * d->g.nb, nnz = 0;
    for (int e = 0; e < d->g.E; ++e) nnz += d->g.nb * (1 + odg_row_count(&d->g, e));

    d->nnz = nnz;
    d->rowptr = malloc(sizeof(int) * (size_t)(N + 1));
    d->col = malloc(sizeof(int) * (size_t)nnz);
    d->val = malloc(sizeof(double) * (size_t)nnz);
    if (!d->rowptr || !d->col || !d->val) return OR_ERR_OOM;
    rc = odg_csr(&d->g, 1, d->rowptr, d->col, d->val);
    if (rc) return rc;
    if (with_air) {
        d->hier = or_air_setup(N, d->rowptr, d->col, d->val, prm, &rc);
        if (rc) return rc;
    }
    return OR_OK;
}

/* Scattering + volumetric source per DOF: (sigma_s phi + q) / (4 pi). */
static void si_source(int E, int nb, const double *sigma_s, const double *q, const double *phi, double *src)
{
    double fourpi = 4.0 * OR_PI;
    for (int e = 0; e < E; ++e)
        for (int a = 0; a < nb; ++a) {
            size_t i = (size_t)e * nb + a;
            src[i] = (sigma_s[e] * phi[i] + q[e]) / fourpi;
        }
}

/* info[0] = SI iterations, info[1] = last relative phi change, info[2] = total
 * inner iterations (V-cycles), info[3] = max final relative inner residual. */
int or_si(const or_mesh *mesh, int M, const double *omega, const double *w, const double *sigma_t,
          const double *sigma_s, const double *q, const or_si_params *sp, const or_params *prm,
          double *phi, double *psi, double *info)
{
    int nb = mesh->kind == 0 ? 8 : 4;
    int E = mesh->kind == 0 ? mesh->n * mesh->n * mesh->n : mesh->T, N = nb * E;
    odir *dirs = calloc(M, sizeof(odir));
    double *src = malloc(sizeof(double) * (size_t)N);
    double *b = malloc(sizeof(double) * (size_t)N);
    double *ginfl = malloc(sizeof(double) * (size_t)N);
    double *phinew = malloc(sizeof(double) * (size_t)N);
    double *srcm = malloc(sizeof(double) * (size_t)N);
    int hmax = sp->inner_cycles > sp->inner_maxit ? sp->inner_cycles : sp->inner_maxit;
    double *hist = malloc(sizeof(double) * (size_t)(hmax + 1));
    int rc = OR_OK;
    if (!dirs || !src || !b || !ginfl || !phinew || !srcm || !hist) { rc = OR_ERR_OOM; goto done; }
    for (int i = 0; i < N; ++i) ginfl[i] = sp->g_inflow;
    for (int m = 0; m < M; ++m) {
        rc = odir_build(&dirs[m], mesh, omega + 3 * m, sigma_t, prm, !sp->use_sweep);
        if (rc) goto done;
    }
    info[0] = 0; info[1] = 0; info[2] = 0; info[3] = 0;
    for (int it = 0; it < sp->max_iters; ++it) {
        si_source(E, nb, sigma_s, q, phi, src);
        for (int i = 0; i < N; ++i) phinew[i] = 0.0;
        for (int m = 0; m < M; ++m) {
            odir *d = &dirs[m];
            const double *sm = src;
            if (sp->q_ang) {
                for (int i = 0; i < N; ++i) srcm[i] = src[i] + sp->q_ang[(size_t)m * N + i];
                sm = srcm;
            }
            odg_rhs(&d->g, sm, sp->g_inflow != 0.0 ? ginfl : NULL, 1, b);
            double *x = psi + (size_t)m * N;
            if (sp->use_sweep) {
                rc = or_sweep(N, nb, d->rowptr, d->col, d->val, b, x, NULL);
                if (rc) goto done;
            } else if (sp->inner_cycles > 0) {
                for (int i = 0; i < N; ++i) x[i] = 0.0;
                int iters = 0;
                or_air_solve(d->hier, b, x, 0.0, sp->inner_cycles, &iters, hist);
                info[2] += iters;
                double bn = norm2(N, b);
                double rel = bn > 0 ? hist[iters] / bn : 0.0;
                if (rel > info[3]) info[3] = rel;
            } else {
                for (int i = 0; i < N; ++i) x[i] = 0.0;
                int iters = 0;
                rc = or_air_solve(d->hier, b, x, sp->inner_tol, sp->inner_maxit, &iters, hist);
                info[2] += iters;
                double bn = norm2(N, b);
                double rel = bn > 0 ? hist[iters] / bn : 0.0;
                if (rel > info[3]) info[3] = rel;
                if (rc) goto done;
            }
            for (int i = 0; i < N; ++i) phinew[i] = phinew[i] + w[m] * x[i];
        }
        double dn = 0.0, pn = 0.0;
        for (int i = 0; i < N; ++i) {
            double t = phinew[i] - phi[i];
            dn = dn + t * t;
            pn = pn + phinew[i] * phinew[i];
        }
        memcpy(phi, phinew, sizeof(double) * (size_t)N);
        info[0] = it + 1;
        info[1] = pn > 0 ? sqrt(dn) / sqrt(pn) : 0.0;
        if (info[1] <= sp->tol) break;
    }
    if (info[1] > sp->tol) rc = OR_ERR_NOT_CONVERGED;
done:
    if (dirs) for (int m = 0; m < M; ++m) odir_free(&dirs[m]);
    free(dirs); free(src); free(b); free(ginfl); free(phinew); free(srcm); free(hist);
    return rc;
}

int or_si_hex(int n, int M, const double *omega, const double *w, const double *sigma_t,
              const double *sigma_s, const double *q, const or_si_params *sp, const or_params *prm,
              double *phi, double *psi, double *info)
{
    or_mesh mesh = {0, n, 0, NULL, NULL, NULL};
    return or_si(&mesh, M, omega, w, sigma_t, sigma_s, q, sp, prm, phi, psi, info);
}

int or_si_tet(int T, const double *verts, const int *tets, const int *nbr, int M, const double *omega,
              const double *w, const double *sigma_t, const double *sigma_s, const double *q,
              const or_si_params *sp, const or_params *prm, double *phi, double *psi, double *info)
{
    or_mesh mesh = {1, 0, T, verts, tets, nbr};
    return or_si(&mesh, M, omega, w, sigma_t, sigma_s, q, sp, prm, phi, psi, info);
}

/* ------------------------------------------------------------------------- */
/* Adjoint source iteration and cross-section gradients (not in the paper).  */
/* Forward: L_m psi_m = M (sigma_s phi + q) / (4 pi), phi = sum_m w_m psi_m,  */
/* J = g^T phi.  Adjoint: L_m^T c_m = phis, phis = g + sigma_s M sum_m w_m    */
/* c_m / (4 pi); with A_m = D_m^{-1} L_m this is A_m^T y_m = phis,            */
/* c_m = D_m^{-T} y_m.  Gradients per element K:                              */
/*   dJ/dsigma_t,K = - sum_m w_m c_{m,K}^T M_K psi_{m,K}                       */
/*   dJ/dsigma_s,K =   sum_m w_m c_{m,K}^T M_K phi_K / (4 pi)                  */
/*   dJ/dq_K       =   sum_m w_m c_{m,K}^T M_K 1 / (4 pi)                      */
/* psi is the converged forward solution (N*M, direction-major).             */
/* info[0] = adjoint SI iterations, info[1] = last relative change.          */
/* ------------------------------------------------------------------------- */
static int or_si_adjoint(const or_mesh *mesh, int M, const double *omega, const double *w,
                         const double *sigma_t, const double *sigma_s, const double *q, const double *psi,
                         const double *g, const or_si_params *sp, const or_params *prm, double *dst, double *dss,
                         double *dq, double *phis, double *info)
{
    int nb = mesh->kind == 0 ? 8 : 4, nn = nb * nb;
    int E = mesh->kind == 0 ? mesh->n * mesh->n * mesh->n : mesh->T, N = nb * E;
    double fourpi = 4.0 * OR_PI;
    odir *dirs = calloc(M, sizeof(odir));
    int **trp = calloc(M, sizeof(int *)), **tci = calloc(M, sizeof(int *));
    double **tv = calloc(M, sizeof(double *));
    void **th = calloc(M, sizeof(void *));
    double *C = malloc(sizeof(double) * (size_t)N * M);   /* c_m = D^{-T} y_m */
    double *acc = malloc(sizeof(double) * (size_t)N);
    double *pnew = malloc(sizeof(double) * (size_t)N);
    double *y = malloc(sizeof(double) * (size_t)N);
    double *phi = calloc(N, sizeof(double));
    double *hist = malloc(sizeof(double) * (size_t)(sp->inner_maxit + 1));
    int rc = OR_OK;
    if (!dirs || !trp || !tci || !tv || !th || !C || !acc || !pnew || !y || !phi || !hist) { rc = OR_ERR_OOM; goto done; }
    for (int m = 0; m < M; ++m) {
        rc = odir_build(&dirs[m], mesh, omega + 3 * m, sigma_t, prm, 0);
        if (rc) goto done;
        rc = csr_transpose(N, dirs[m].rowptr, dirs[m].col, dirs[m].val, &trp[m], &tci[m], &tv[m]);
        if (rc) goto done;
        if (!sp->use_sweep) {
            th[m] = or_air_setup(N, trp[m], tci[m], tv[m], prm, &rc);
            if (rc) goto done;
        }
        for (int i = 0; i < N; ++i) phi[i] = phi[i] + w[m] * psi[(size_t)m * N + i];
    }
    for (int i = 0; i < N; ++i) phis[i] = 0.0;
    info[0] = 0; info[1] = 0;
    for (int it = 0; it < sp->max_iters; ++it) {
        for (int i = 0; i < N; ++i) acc[i] = 0.0;
        for (int m = 0; m < M; ++m) {
            odg *gd = &dirs[m].g;
            if (sp->use_sweep) {
                rc = or_sweep_scc(N, nb, trp[m], tci[m], tv[m], phis, y, NULL, NULL);
                if (rc) goto done;
            } else {
                for (int i = 0; i < N; ++i) y[i] = 0.0;
                int iters = 0;
                rc = or_air_solve(th[m], phis, y, sp->inner_tol, sp->inner_maxit, &iters, hist);
                if (rc && rc != OR_ERR_NOT_CONVERGED) goto done;
                rc = OR_OK;
            }
            double *c = C + (size_t)m * N;
            for (int e = 0; e < E; ++e) {
                memcpy(c + nb * e, y + nb * e, sizeof(double) * nb);
                lu_solve_transpose(nb, gd->D + (size_t)e * nn, gd->piv + (size_t)e * nb, c + nb * e);
                const double *Mk = gd->Mass + (size_t)e * nn;
                for (int a = 0; a < nb; ++a) {
                    double s = 0.0;
                    for (int b = 0; b < nb; ++b) s = s + Mk[a * nb + b] * c[nb * e + b];
                    acc[nb * e + a] = acc[nb * e + a] + w[m] * s;
                }
            }
        }
        double dn = 0.0, pn = 0.0;
        for (int e = 0; e < E; ++e)
            for (int a = 0; a < nb; ++a) {
                int i = nb * e + a;
                pnew[i] = g[i] + sigma_s[e] * acc[i] / fourpi;
                double t = pnew[i] - phis[i];
                dn = dn + t * t;
                pn = pn + pnew[i] * pnew[i];
            }
        memcpy(phis, pnew, sizeof(double) * (size_t)N);
        info[0] = it + 1;
        info[1] = pn > 0 ? sqrt(dn) / sqrt(pn) : 0.0;
        if (info[1] <= sp->tol) break;
    }
    /* gradients with the last adjoint solutions */
    for (int e = 0; e < E; ++e) { dst[e] = 0.0; dss[e] = 0.0; dq[e] = 0.0; }
    for (int m = 0; m < M; ++m) {
        const double *c = C + (size_t)m * N;
        const double *ps = psi + (size_t)m * N;
        odg *gd = &dirs[m].g;
        for (int e = 0; e < E; ++e) {
            const double *Mk = gd->Mass + (size_t)e * nn;
            double t_psi = 0.0, t_phi = 0.0, t_one = 0.0;
            for (int a = 0; a < nb; ++a) {
                double mp = 0.0, mf = 0.0, m1 = 0.0;
                for (int b = 0; b < nb; ++b) {
                    mp = mp + Mk[a * nb + b] * ps[nb * e + b];
                    mf = mf + Mk[a * nb + b] * phi[nb * e + b];
                    m1 = m1 + Mk[a * nb + b];
                }
                t_psi = t_psi + c[nb * e + a] * mp;
                t_phi = t_phi + c[nb * e + a] * mf;
                t_one = t_one + c[nb * e + a] * m1;
            }
            dst[e] = dst[e] - w[m] * t_psi;
            dss[e] = dss[e] + w[m] * t_phi / fourpi;
            dq[e] = dq[e] + w[m] * t_one / fourpi;
        }
    }
    if (info[1] > sp->tol && sp->max_iters > 1) rc = OR_ERR_NOT_CONVERGED;
done:
    if (dirs) for (int m = 0; m < M; ++m) odir_free(&dirs[m]);
    if (trp) for (int m = 0; m < M; ++m) { free(trp[m]); free(tci[m]); free(tv[m]); if (th[m]) or_hier_free(th[m]); }
    free(dirs); free(trp); free(tci); free(tv); free(th); free(C); free(acc); free(pnew); free(y); free(phi); free(hist);
    return rc;
}

int or_si_adjoint_hex(int n, int M, const double *omega, const double *w, const double *sigma_t,
                      const double *sigma_s, const double *q, const double *psi, const double *g,
                      const or_si_params *sp, const or_params *prm, double *dst, double *dss, double *dq,
                      double *phis, double *info)
{
    or_mesh mesh = {0, n, 0, NULL, NULL, NULL};
    return or_si_adjoint(&mesh, M, omega, w, sigma_t, sigma_s, q, psi, g, sp, prm, dst, dss, dq, phis, info);
}

int or_si_adjoint_tet(int T, const double *verts, const int *tets, const int *nbr, int M, const double *omega,
                      const double *w, const double *sigma_t, const double *sigma_s, const double *q,
                      const double *psi, const double *g, const or_si_params *sp, const or_params *prm,
                      double *dst, double *dss, double *dq, double *phis, double *info)
{
    or_mesh mesh = {1, 0, T, verts, tets, nbr};
    return or_si_adjoint(&mesh, M, omega, w, sigma_t, sigma_s, q, psi, g, sp, prm, dst, dss, dq, phis, info);
}
