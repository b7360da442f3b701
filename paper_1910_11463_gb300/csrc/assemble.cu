// Upwind DG assembly on the structured hex Q1 mesh with block-inverse scaling
// (Eq. weak_form_transport; Sec. 1.3).  Compiled with --fmad=false: every
// product and sum below is rounded as written, in the order written (fused
// multiply-adds only where fma() is written), so the scaled operator is
// reproducible bit for bit.
//
// One thread per (element, direction).  Per element K and direction Omega:
//   m1[i][j] = (2 or 1) h / 6,  g1[i][j] = -1/2 (i = 0), +1/2 (i = 1)
//   L_KK[a][b] = sigma_t mass(a,b) - ((mu gx + eta gy) + xi gz)
//                + |Omega_d| face_d(a,b)   on each outflow face (both nodes on it)
//   L_KK'[a][b] = -|Omega_d| face_d(a,b)   a on K's inflow face, b on K''s face
// L_KK is factored by LU with partial pivoting; the stored blocks are
// D_K^{-1} L_KK' (8 x 4, the four columns of the upwind element's face nodes)
// and W_K = D_K^{-1} M_K (8 x 8, for right-hand sides).
#include "common.cuh"

namespace pr {

namespace {

// LU with partial pivoting (first maximum), multipliers a_rk * (1 / a_kk),
// updates fma(-l, a_kc, a_rc); column-oriented substitutions with fma and
// y_k * (1 / u_kk).  The same operation sequence as every LU in the library.
template <int n>
__device__ __forceinline__ void lu_factorN(double *a, int *piv, double *rinv, int *singular) {
    for (int k = 0; k < n; ++k) {
        int p = k;
        long long mx = absbits(a[k * n + k]);
        for (int r = k + 1; r < n; ++r) {
            long long v = absbits(a[r * n + k]);
            if (v > mx) { mx = v; p = r; }
        }
        piv[k] = p;
        if (!(mx > 0)) { *singular = 1; return; }
        if (p != k)
            for (int c = 0; c < n; ++c) { double t = a[k * n + c]; a[k * n + c] = a[p * n + c]; a[p * n + c] = t; }
        double rd = 1.0 / a[k * n + k];
        rinv[k] = rd;   // row k is final from here on: the back substitution reuses it
        for (int r = k + 1; r < n; ++r) {
            double l = a[r * n + k] * rd;
            a[r * n + k] = l;
            for (int c = k + 1; c < n; ++c) a[r * n + c] = fma(-l, a[k * n + c], a[r * n + c]);
        }
    }
}

template <int n>
__device__ __forceinline__ void lu_solveN(const double *a, const int *piv, const double *rinv, double *y) {
    for (int k = 0; k < n; ++k)
        if (piv[k] != k) { double t = y[k]; y[k] = y[piv[k]]; y[piv[k]] = t; }
    for (int k = 0; k < n; ++k)
        for (int r = k + 1; r < n; ++r) y[r] = fma(-a[r * n + k], y[k], y[r]);
    for (int k = n - 1; k >= 0; --k) {
        y[k] = y[k] * rinv[k];
        for (int r = 0; r < k; ++r) y[r] = fma(-a[r * n + k], y[k], y[r]);
    }
}

struct HexFactors {
    double m1[2][2];
};

__device__ __forceinline__ double face_f(const double (*m1)[2], int d, int a, int b) {
    int ax = a & 1, ay = (a >> 1) & 1, az = (a >> 2) & 1;
    int bx = b & 1, by = (b >> 1) & 1, bz = (b >> 2) & 1;
    return (d == 0) ? m1[ay][by] * m1[az][bz] : (d == 1) ? m1[ax][bx] * m1[az][bz] : m1[ax][bx] * m1[ay][by];
}

// rows of element e in direction m: 8 * (1 + 4 * upwind neighbours)
__global__ void k_hex_rowcounts(int n, int ndir, const double *omega, int *counts) {
    long long E = (long long)n * n * n;
    long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= E * ndir) return;
    int m = (int)(tid / E);
    int e = (int)(tid % E);
    int idx[3] = {e % n, (e / n) % n, e / (n * n)};
    int c = 1;
    for (int d = 0; d < 3; ++d) {
        double o = omega[3 * m + d];
        if (o == 0.0) continue;
        if (o > 0.0 ? idx[d] > 0 : idx[d] < n - 1) c += 4;
    }
    long long r0 = (long long)m * 8 * E + 8LL * e;
    for (int a = 0; a < 8; ++a) counts[r0 + a] = c;
}

__global__ void __launch_bounds__(128) k_hex_assemble(int n, int ndir, const double *omega, const double *sigma_t,
                                                      const int *rowptr, int *col, double *val, double *bsr64,
                                                      float *bsr32, double *W, double *Gin, int *err) {
    long long E = (long long)n * n * n;
    long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= E * ndir) return;
    int m = (int)(tid / E);
    int e = (int)(tid % E);
    const double om[3] = {omega[3 * m], omega[3 * m + 1], omega[3 * m + 2]};
    double h = 1.0 / (double)n;
    double m1[2][2];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) m1[i][j] = ((i == j) ? 2.0 : 1.0) * h / 6.0;
    const double g1[2][2] = {{-0.5, -0.5}, {0.5, 0.5}};
    int out[3], in[3];
    for (int d = 0; d < 3; ++d) { out[d] = om[d] > 0.0 ? 1 : 0; in[d] = 1 - out[d]; }
    double st = sigma_t[e];
    double D[64];
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
            D[a * 8 + b] = v;
        }
    }
    int piv[8];
    double rinv[8];
    int sing = 0;
    lu_factorN<8>(D, piv, rinv, &sing);
    if (sing) { atomicOr(err, 1); return; }

    int idx[3] = {e % n, (e / n) % n, e / (n * n)};
    const int stride[3] = {1, n, n * n};
    // upwind neighbours (element, axis), sorted by element index with e itself
    int nb_e[4], nb_d[4], cnt = 0;
    for (int d = 0; d < 3; ++d) {
        if (om[d] == 0.0) continue;
        bool has = om[d] > 0.0 ? idx[d] > 0 : idx[d] < n - 1;
        if (!has) continue;
        nb_e[cnt] = om[d] > 0.0 ? e - stride[d] : e + stride[d];
        nb_d[cnt] = d;
        ++cnt;
    }
    nb_e[cnt] = e;
    nb_d[cnt] = -1;
    int tot = cnt + 1;
    for (int i = 1; i < tot; ++i)
        for (int j = i; j > 0 && nb_e[j - 1] > nb_e[j]; --j) {
            int t = nb_e[j]; nb_e[j] = nb_e[j - 1]; nb_e[j - 1] = t;
            t = nb_d[j]; nb_d[j] = nb_d[j - 1]; nb_d[j - 1] = t;
        }
    double Y[3][4][8];   // [axis][face node][row]
    bool hasax[3] = {false, false, false};
    for (int k = 0; k < tot; ++k) {
        int d = nb_d[k];
        if (d < 0) continue;
        hasax[d] = true;
        double w = fabs(om[d]);
        int t = 0;
        for (int b = 0; b < 8; ++b) {
            if (((b >> d) & 1) != out[d]) continue;
            double *y = Y[d][t];
            for (int a = 0; a < 8; ++a) y[a] = (((a >> d) & 1) != in[d]) ? 0.0 : -(w * face_f(m1, d, a, b));
            lu_solveN<8>(D, piv, rinv, y);
            ++t;
        }
    }
    long long N = 8 * E;
    long long rowbase = (long long)m * N + 8LL * e;
    if (col) {
        for (int a = 0; a < 8; ++a) {
            long long p = rowptr[rowbase + a];
            for (int k = 0; k < tot; ++k) {
                int d = nb_d[k];
                if (d < 0) {
                    col[p] = (int)(rowbase + a);
                    val[p] = 1.0;
                    ++p;
                    continue;
                }
                int t = 0;
                for (int b = 0; b < 8; ++b) {
                    if (((b >> d) & 1) != out[d]) continue;
                    col[p] = (int)((long long)m * N + 8LL * nb_e[k] + b);
                    val[p] = Y[d][t][a];
                    ++p;
                    ++t;
                }
            }
        }
    }
    if (bsr64 || bsr32) {
        long long base = ((long long)m * E + e) * 3;
        for (int d = 0; d < 3; ++d)
            for (int a = 0; a < 8; ++a)
                for (int t = 0; t < 4; ++t) {
                    double v = hasax[d] ? Y[d][t][a] : 0.0;
                    if (bsr64) bsr64[(base + d) * 32 + a * 4 + t] = v;
                    if (bsr32) bsr32[(base + d) * 32 + a * 4 + t] = (float)v;
                }
    }
    if (Gin) {
        // D_K^{-1} sum over boundary inflow faces of |Omega_d| int_F phi_b phi_a (unit inflow)
        double y[8];
        for (int a = 0; a < 8; ++a) {
            double acc = 0.0;
            for (int d = 0; d < 3; ++d) {
                if (om[d] == 0.0) continue;
                bool bnd = om[d] > 0.0 ? idx[d] == 0 : idx[d] == n - 1;
                if (!bnd || ((a >> d) & 1) != in[d]) continue;
                double w = fabs(om[d]), s = 0.0;
                for (int b = 0; b < 8; ++b)
                    if (((b >> d) & 1) == in[d]) s = s + w * face_f(m1, d, a, b);
                acc = acc + s;
            }
            y[a] = acc;
        }
        lu_solveN<8>(D, piv, rinv, y);
        for (int a = 0; a < 8; ++a) Gin[((long long)m * E + e) * 8 + a] = y[a];
    }
    if (W) {
        double *We = W + ((long long)m * E + e) * 64;
        for (int b = 0; b < 8; ++b) {
            int bx = b & 1, by = (b >> 1) & 1, bz = (b >> 2) & 1;
            double y[8];
            for (int a = 0; a < 8; ++a) {
                int ax = a & 1, ay = (a >> 1) & 1, az = (a >> 2) & 1;
                y[a] = (m1[ax][bx] * m1[ay][by]) * m1[az][bz];
            }
            lu_solveN<8>(D, piv, rinv, y);
            for (int a = 0; a < 8; ++a) We[a * 8 + b] = y[a];
        }
    }
}


// ---- tetrahedra, P1 -----------------------------------------------------------
// Local node a = tet vertex a; face f = the triangle without vertex f.
// e_k = x_k - x_0; c23 = e2 x e3, c31 = e3 x e1, c12 = e1 x e2; det = e1 . c23;
// grad l1 = c23 / det, grad l2 = c31 / det, grad l3 = c12 / det,
// grad l0 = -((grad l1 + grad l2) + grad l3); |K| = |det| / 6; od_a = Omega . grad l_a;
// face flux (Omega.n)|F| = -(od_f (3 |K|)).
// L_KK[a][b] = sigma_t (c_ab |K| / 20) - (od_a |K|) / 4 + sum_{outflow f, a,b != f} (fl_f c_ab) / 12
// L_KK'[a][b'] = (fl_f c) / 12 on the inflow face f (c = 2 on the same vertex, else 1).
struct TetGeom {
    double od[4], fl[4], vol;
};

__device__ __forceinline__ void cross3(const double *a, const double *b, double *c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
__device__ __forceinline__ double dot3(const double *a, const double *b) { return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2]; }

__device__ __forceinline__ bool tet_geom(const double *verts, const int *tv, const double *om, TetGeom &g) {
    double x[4][3], e[3][3], gr[4][3], c23[3], c31[3], c12[3];
    for (int a = 0; a < 4; ++a)
        for (int k = 0; k < 3; ++k) x[a][k] = verts[3 * tv[a] + k];
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k) e[j][k] = x[j + 1][k] - x[0][k];
    cross3(e[1], e[2], c23);
    cross3(e[2], e[0], c31);
    cross3(e[0], e[1], c12);
    double det = dot3(e[0], c23);
    if (det == 0.0) return false;
    for (int k = 0; k < 3; ++k) {
        gr[1][k] = c23[k] / det;
        gr[2][k] = c31[k] / det;
        gr[3][k] = c12[k] / det;
        gr[0][k] = -((gr[1][k] + gr[2][k]) + gr[3][k]);
    }
    g.vol = fabs(det) / 6.0;
    for (int a = 0; a < 4; ++a) g.od[a] = dot3(om, gr[a]);
    for (int f = 0; f < 4; ++f) g.fl[f] = -(g.od[f] * (3.0 * g.vol));
    return true;
}

__global__ void k_tet_rowcounts(int T, int ndir, const double *omega, const double *verts, const int *tets,
                                const int *nbr, int *counts) {
    long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (long long)T * ndir) return;
    int m = (int)(tid / T), t = (int)(tid % T);
    const double om[3] = {omega[3 * m], omega[3 * m + 1], omega[3 * m + 2]};
    TetGeom g;
    int c = 1;
    if (tet_geom(verts, tets + 4 * t, om, g))
        for (int f = 0; f < 4; ++f)
            if (g.fl[f] < 0.0 && nbr[4 * t + f] >= 0) c += 3;
    long long r0 = ((long long)m * T + t) * 4;
    for (int a = 0; a < 4; ++a) counts[r0 + a] = c;
}

__global__ void __launch_bounds__(128) k_tet_assemble(int T, int ndir, const double *omega, const double *verts,
                                                      const int *tets, const int *nbr, const double *sigma_t,
                                                      const int *rowptr, int *col, double *val, double *W,
                                                      double *Gin, int *err) {
    long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (long long)T * ndir) return;
    int m = (int)(tid / T), t = (int)(tid % T);
    const double om[3] = {omega[3 * m], omega[3 * m + 1], omega[3 * m + 2]};
    const int *tv = tets + 4 * t;
    TetGeom g;
    if (!tet_geom(verts, tv, om, g)) { atomicOr(err, 1); return; }
    double st = sigma_t[t], vol = g.vol;
    double D[16];
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            double mass = ((a == b) ? 2.0 : 1.0) * vol / 20.0;
            double v = st * mass - g.od[a] * vol / 4.0;
            for (int f = 0; f < 4; ++f) {
                if (!(g.fl[f] > 0.0) || a == f || b == f) continue;
                v = v + g.fl[f] * ((a == b) ? 2.0 : 1.0) / 12.0;
            }
            D[a * 4 + b] = v;
        }
    int piv[4], sing = 0;
    double rinv[4];
    lu_factorN<4>(D, piv, rinv, &sing);
    if (sing) { atomicOr(err, 1); return; }
    // inflow faces with an upwind neighbour, sorted by neighbour index with t itself
    int nb_e[5], nb_f[5], cnt = 0;
    for (int f = 0; f < 4; ++f)
        if (g.fl[f] < 0.0 && nbr[4 * t + f] >= 0) { nb_e[cnt] = nbr[4 * t + f]; nb_f[cnt] = f; ++cnt; }
    nb_e[cnt] = t;
    nb_f[cnt] = -1;
    int tot = cnt + 1;
    for (int i = 1; i < tot; ++i)
        for (int j = i; j > 0 && nb_e[j - 1] > nb_e[j]; --j) {
            int x = nb_e[j]; nb_e[j] = nb_e[j - 1]; nb_e[j - 1] = x;
            x = nb_f[j]; nb_f[j] = nb_f[j - 1]; nb_f[j - 1] = x;
        }
    double Y[4][3][4];   // [face][face node][row]
    int Ynode[4][3];
    for (int k = 0; k < tot; ++k) {
        int f = nb_f[k];
        if (f < 0) continue;
        const int *uv = tets + 4 * nb_e[k];
        int u = 0;
        for (int b = 0; b < 4 && u < 3; ++b) {
            bool onface = false;
            for (int a = 0; a < 4; ++a)
                if (a != f && tv[a] == uv[b]) onface = true;
            if (!onface) continue;
            Ynode[f][u] = b;
            double *y = Y[f][u];
            for (int a = 0; a < 4; ++a) y[a] = (a == f) ? 0.0 : g.fl[f] * ((tv[a] == uv[b]) ? 2.0 : 1.0) / 12.0;
            lu_solveN<4>(D, piv, rinv, y);
            ++u;
        }
        if (u != 3) atomicOr(err, 2);
    }
    long long N = 4LL * T;
    long long rowbase = (long long)m * N + 4LL * t;
    if (col) {
        for (int a = 0; a < 4; ++a) {
            long long p = rowptr[rowbase + a];
            for (int k = 0; k < tot; ++k) {
                int f = nb_f[k];
                if (f < 0) { col[p] = (int)(rowbase + a); val[p] = 1.0; ++p; continue; }
                for (int u = 0; u < 3; ++u) {
                    col[p] = (int)((long long)m * N + 4LL * nb_e[k] + Ynode[f][u]);
                    val[p] = Y[f][u][a];
                    ++p;
                }
            }
        }
    }
    if (Gin) {
        // D^{-1} (boundary inflow faces: sum_b |fl_f| c_ab / 12, unit inflow)
        double y[4];
        for (int a = 0; a < 4; ++a) {
            double acc = 0.0;
            for (int f = 0; f < 4; ++f) {
                if (!(g.fl[f] < 0.0) || nbr[4 * t + f] >= 0 || a == f) continue;
                double s2 = 0.0;
                for (int b = 0; b < 4; ++b)
                    if (b != f) s2 = s2 + -(g.fl[f] * ((a == b) ? 2.0 : 1.0) / 12.0);
                acc = acc + s2;
            }
            y[a] = acc;
        }
        lu_solveN<4>(D, piv, rinv, y);
        for (int a = 0; a < 4; ++a) Gin[((long long)m * T + t) * 4 + a] = y[a];
    }
    if (W) {
        double *We = W + ((long long)m * T + t) * 16;
        for (int b = 0; b < 4; ++b) {
            double y[4];
            for (int a = 0; a < 4; ++a) y[a] = ((a == b) ? 2.0 : 1.0) * vol / 20.0;
            lu_solveN<4>(D, piv, rinv, y);
            for (int a = 0; a < 4; ++a) We[a * 4 + b] = y[a];
        }
    }
}

}  // namespace

// Assembles 'ndir' directions (omega: device [ndir][3]).  Any output may be
// null.  CSR: rowptr (ndir * 8 n^3 + 1), col/val (hex_nnz entries), rows and
// columns offset by m * 8 n^3.  Block form: bsr64/bsr32 [dir][elem][axis][a][4].
// W [dir][elem][8][8] = D^{-1} M.  Gin [dir][N] = D^{-1} (unit boundary inflow).
void hex_assemble(int n, int ndir, const double *omega_d, const double *sigma_t, int *rowptr, int *col,
                  double *val, double *bsr64, float *bsr32, double *W, double *Gin, int *d_err, cudaStream_t s) {
    long long E = (long long)n * n * n;
    long long rows = 8 * E * ndir;
    PR_REQUIRE(rows < 0x7fffffffLL, PAIR_ERR_UNSUPPORTED, "hex batch has more than 2^31 rows");
    if (rowptr) {
        int *counts = dmalloc<int>(rows, s);
        k_hex_rowcounts<<<blocks_for(E * ndir, 256), 256, 0, s>>>(n, ndir, omega_d, counts);
        PR_LAUNCH();
        scan_exclusive(counts, rowptr, (int)rows, s, false);
        dfree(counts, s);
    }
    k_hex_assemble<<<blocks_for(E * ndir, 128), 128, 0, s>>>(n, ndir, omega_d, sigma_t, rowptr, col, val, bsr64,
                                                              bsr32, W, Gin, d_err);
    PR_LAUNCH();
}

// Tetrahedral mesh, 'ndir' directions: CSR (rows/cols offset by m * 4T), W
// [dir][tet][4][4] = D^{-1} M, Gin [dir][4T].  Computes rowptr; returns nnz.
long long tet_assemble(int T, int ndir, const double *omega_d, const double *verts, const int *tets, const int *nbr,
                       const double *sigma_t, int *rowptr, int *col, double *val, double *W, double *Gin, int *d_err,
                       cudaStream_t s, bool rowptr_only) {
    long long rows = 4LL * T * ndir;
    PR_REQUIRE(rows < 0x7fffffffLL, PAIR_ERR_UNSUPPORTED, "tet batch has more than 2^31 rows");
    int *counts = dmalloc<int>(rows, s);
    k_tet_rowcounts<<<blocks_for((long long)T * ndir, 256), 256, 0, s>>>(T, ndir, omega_d, verts, tets, nbr, counts);
    PR_LAUNCH();
    long long nnz = scan_exclusive(counts, rowptr, (int)rows, s);
    dfree(counts, s);
    if (rowptr_only) return nnz;
    k_tet_assemble<<<blocks_for((long long)T * ndir, 128), 128, 0, s>>>(T, ndir, omega_d, verts, tets, nbr, sigma_t,
                                                                        rowptr, col, val, W, Gin, d_err);
    PR_LAUNCH();
    return nnz;
}

// Stored entries of the scaled operator of one direction (closed form).
long long hex_nnz(int n, const double *omega_h) {
    long long E = (long long)n * n * n, nnz = 8 * E;
    for (int d = 0; d < 3; ++d)
        if (omega_h[d] != 0.0) nnz += 32LL * n * n * (n - 1);
    return nnz;
}

}  // namespace pr
