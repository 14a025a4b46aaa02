/*
 * fegen.c -- seeded synthetic finite-element stiffness matrices (input generator).
 *
 * This file builds the INPUTS that both the CPU oracle and the CUDA library
 * consume: P1 tetrahedral stiffness matrices on structured, jittered, randomly
 * renumbered node grids.  It holds none of the arithmetic of the method under
 * test (no sparse matrix-vector product, no conjugate gradient); all random
 * numbers are drawn by the Python side (numpy PCG64) and passed in.
 *
 * Discretisation (paper Sec. 2): isoparametric linear tetrahedra with one
 * integration point, i.e. element matrices K_e = V_e * G^T D G for the
 * diffusion operator div(D grad phi), D = d_iso I + d_ani n (x) n.  The linear
 * elasticity variant uses K_e = V_e * B^T C B with an isotropic C(E, nu).
 *
 * Mesh: an n0 x n1 x n2 node grid (axis 2 optionally periodic), every hex cell
 * split into 6 tetrahedra along its (0,0,0)-(1,1,1) diagonal (Kuhn split), so
 * each interior node couples to 14 neighbours plus itself.
 *
 * Compile with -ffp-contract=off so that the element arithmetic is identical
 * on every host.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define FEGEN_MAX_DEG 32

/* The 6 axis orders of the Kuhn split; tet = {0, e_a, e_a+e_b, 1}. */
static const int kuhn_perm[6][3] = {
    {0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
/* parity (+1 even, -1 odd) of each axis order */
static const int kuhn_sign[6] = {+1, -1, -1, +1, +1, -1};

static int64_t grid_id(int64_t i0, int64_t i1, int64_t i2, int n1, int n2) {
    return (i0 * n1 + i1) * n2 + i2;
}

/* The four grid ids of tet t of cell (c0,c1,c2). */
static void tet_nodes(int c0, int c1, int c2, int t, int n1, int n2, int periodic2,
                      int64_t out[4]) {
    int v[3] = {c0, c1, c2};
    int w[3];
    for (int k = 0; k < 4; ++k) {
        w[0] = v[0]; w[1] = v[1]; w[2] = v[2];
        for (int s = 0; s < k && s < 3; ++s) w[kuhn_perm[t][s]] += 1;
        if (k == 3) { w[0] = v[0] + 1; w[1] = v[1] + 1; w[2] = v[2] + 1; }
        if (periodic2 && w[2] == n2) w[2] = 0;
        out[k] = grid_id(w[0], w[1], w[2], n1, n2);
    }
}

static int64_t n_cells2(int n2, int periodic2) { return periodic2 ? n2 : n2 - 1; }

/* Kuhn neighbours of a grid node: the 14 offsets of the split plus the node itself. */
static const int kuhn_nbr[15][3] = {
    {0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {0, 1, 1}, {0, -1, -1}, {1, 0, 1}, {-1, 0, -1}, {1, 1, 1}, {-1, -1, -1}};

/* Node adjacency (new numbering, self included, ascending) of every node, built
 * from the split's edge offsets; nodes are independent, so rows run in parallel. */
static int build_adjacency(int n0, int n1, int n2, int periodic2, const int32_t* newid,
                           int32_t* deg, int32_t* adj /* n_nodes*FEGEN_MAX_DEG */) {
    int64_t nn = (int64_t)n0 * n1 * n2;
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < nn; ++g) {
        int i0 = (int)(g / ((int64_t)n1 * n2)), i1 = (int)((g / n2) % n1), i2 = (int)(g % n2);
        int32_t a = newid[g];
        int32_t* row = adj + (int64_t)a * FEGEN_MAX_DEG;
        int d = 0;
        for (int k = 0; k < 15; ++k) {
            int j0 = i0 + kuhn_nbr[k][0], j1 = i1 + kuhn_nbr[k][1], j2 = i2 + kuhn_nbr[k][2];
            if (j0 < 0 || j0 >= n0 || j1 < 0 || j1 >= n1) continue;
            if (periodic2) {
                j2 = (j2 + n2) % n2;
            } else if (j2 < 0 || j2 >= n2) {
                continue;
            }
            int32_t v = newid[grid_id(j0, j1, j2, n1, n2)];
            int dup = 0;
            for (int q = 0; q < d; ++q)
                if (row[q] == v) dup = 1;
            if (!dup) row[d++] = v;
        }
        for (int i = 1; i < d; ++i) {   /* insertion sort, <= 15 entries */
            int32_t v = row[i];
            int j = i - 1;
            while (j >= 0 && row[j] > v) { row[j + 1] = row[j]; --j; }
            row[j + 1] = v;
        }
        deg[a] = d;
    }
    return 0;
}

/* Degrees (self included) of every node in the new numbering. */
int fegen_node_degrees(int n0, int n1, int n2, int periodic2, const int32_t* newid,
                       int32_t* deg) {
    int64_t nn = (int64_t)n0 * n1 * n2;
    int32_t* adj = (int32_t*)malloc((size_t)nn * FEGEN_MAX_DEG * sizeof(int32_t));
    if (!adj) return -2;
    int rc = build_adjacency(n0, n1, n2, periodic2, newid, deg, adj);
    free(adj);
    return rc;
}

/* 3x3 inverse-transpose rows: gradients of the barycentric functions. */
static double tet_gradients(const double x[4][3], double g[4][3]) {
    double J[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) J[r][c] = x[c + 1][r] - x[0][r]; /* columns = edges */
    double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1])
               - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0])
               + J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    double inv[3][3];
    inv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
    inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    inv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
    inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    inv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
    inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    /* grad N_a (a=1..3) is row a-1 of J^{-1}; grad N_0 = -(sum of the others) */
    for (int a = 1; a < 4; ++a)
        for (int d = 0; d < 3; ++d) g[a][d] = inv[a - 1][d];
    for (int d = 0; d < 3; ++d) g[0][d] = -(g[1][d] + g[2][d] + g[3][d]);
    return det;
}

static int32_t find_col(const int32_t* row, int deg, int32_t col) {
    for (int k = 0; k < deg; ++k)
        if (row[k] == col) return k;
    return -1;
}

/* Element matrix of one tet (ne = 4 or 12 rows, full symmetric storage); returns
 * det * parity (its sign is the tet's orientation) or 0 for a degenerate tet. */
static double element_matrix(int kind, const double x[4][3], const double* fib, double E,
                             double d_iso, double d_ani, double nu, int t, double* Ke) {
    double gr[4][3];
    double det = tet_gradients(x, gr);
    if (!(det != 0.0) || !isfinite(det)) return 0.0;
    double vol = fabs(det) / 6.0;
    if (kind != 2) {
        double D[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
        if (kind == 1)
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    D[i][j] = (i == j ? d_iso : 0.0) + d_ani * fib[i] * fib[j];
        for (int a = 0; a < 4; ++a) {
            double Dg[3];
            for (int i = 0; i < 3; ++i)
                Dg[i] = D[i][0] * gr[a][0] + D[i][1] * gr[a][1] + D[i][2] * gr[a][2];
            for (int b = a; b < 4; ++b) {
                double v = vol * (gr[b][0] * Dg[0] + gr[b][1] * Dg[1] + gr[b][2] * Dg[2]);
                Ke[a * 4 + b] = v;
                Ke[b * 4 + a] = v;
            }
        }
    } else {
        double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
        double mu = E / (2.0 * (1.0 + nu));
        double B[6][12];
        memset(B, 0, sizeof(B));
        for (int a = 0; a < 4; ++a) {
            double gx = gr[a][0], gy = gr[a][1], gz = gr[a][2];
            B[0][3 * a + 0] = gx;
            B[1][3 * a + 1] = gy;
            B[2][3 * a + 2] = gz;
            B[3][3 * a + 1] = gz; B[3][3 * a + 2] = gy;
            B[4][3 * a + 0] = gz; B[4][3 * a + 2] = gx;
            B[5][3 * a + 0] = gy; B[5][3 * a + 1] = gx;
        }
        double C[6][6];
        memset(C, 0, sizeof(C));
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) C[i][j] = lam + (i == j ? 2.0 * mu : 0.0);
        C[3][3] = C[4][4] = C[5][5] = mu;
        double CB[6][12];
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 12; ++j) {
                double s2 = 0.0;
                for (int k = 0; k < 6; ++k) s2 += C[i][k] * B[k][j];
                CB[i][j] = s2;
            }
        for (int i = 0; i < 12; ++i)
            for (int j = i; j < 12; ++j) {
                double s2 = 0.0;
                for (int k = 0; k < 6; ++k) s2 += B[k][i] * CB[k][j];
                Ke[i * 12 + j] = vol * s2;
                Ke[j * 12 + i] = Ke[i * 12 + j];
            }
    }
    return det * kuhn_sign[t];
}

/* Position (0..3) of grid node g among the vertices of tet t of cell (c0,c1,c2), or -1. */
static int local_vertex(int c0, int c1, int c2, int t, int n1, int n2, int periodic2, int64_t g) {
    int64_t v[4];
    tet_nodes(c0, c1, c2, t, n1, n2, periodic2, v);
    for (int k = 0; k < 4; ++k)
        if (v[k] == g) return k;
    return -1;
}

/*
 * Assemble the stiffness matrix in the new numbering.
 *   kind 0: scalar diffusion, D = I
 *   kind 1: scalar diffusion, D = d_iso I + d_ani n n^T, n = coef[3*cell .. 3*cell+2]
 *   kind 2: linear elasticity, 3 dof/node (dof = 3*node + c), E = coef[tet], Poisson nu
 * xyz: physical node coordinates in grid order (3 per node).
 * rowptr/colind/values: sized from fegen_node_degrees (rows = dofs); colind sorted.
 * Element matrices are computed once per tet (in parallel); each row then sums
 * the contributions of its incident tets in ascending tet order (rows in
 * parallel), which is the order of a sequential loop over tets, so the result
 * does not depend on the thread count and A is bitwise symmetric.
 * Returns 0, -1 (adjacency overflow), -2 (alloc), -3 (inverted or degenerate tet).
 * bad_tet receives the id of the first inverted tet when -3 is returned.
 */
int fegen_assemble(int kind, int n0, int n1, int n2, int periodic2, const double* xyz,
                   const int32_t* newid, const double* coef, double d_iso, double d_ani,
                   double nu, int64_t* rowptr, int32_t* colind, double* values,
                   int64_t* bad_tet) {
    int64_t nn = (int64_t)n0 * n1 * n2;
    int dpn = (kind == 2) ? 3 : 1;
    int ne = 4 * dpn;
    int64_t nc2 = n_cells2(n2, periodic2);
    int64_t ncells = (int64_t)(n0 - 1) * (n1 - 1) * nc2;
    int64_t ntets = ncells * 6;
    int32_t* deg = (int32_t*)malloc((size_t)nn * sizeof(int32_t));
    int32_t* adj = (int32_t*)malloc((size_t)nn * FEGEN_MAX_DEG * sizeof(int32_t));
    double* Ke = (double*)malloc((size_t)(ntets > 0 ? ntets : 1) * ne * ne * sizeof(double));
    signed char* orient = (signed char*)malloc((size_t)(ntets > 0 ? ntets : 1));
    if (!deg || !adj || !Ke || !orient) { free(deg); free(adj); free(Ke); free(orient); return -2; }
    int rc = build_adjacency(n0, n1, n2, periodic2, newid, deg, adj);
    if (rc) { free(deg); free(adj); free(Ke); free(orient); return rc; }

    /* 1. element matrices, one per tet */
#pragma omp parallel for schedule(static)
    for (int64_t cell = 0; cell < ncells; ++cell) {
        int c0 = (int)(cell / ((int64_t)(n1 - 1) * nc2));
        int c1 = (int)((cell / nc2) % (n1 - 1));
        int c2 = (int)(cell % nc2);
        for (int t = 0; t < 6; ++t) {
            int64_t tet = cell * 6 + t;
            int64_t g[4];
            double x[4][3];
            tet_nodes(c0, c1, c2, t, n1, n2, periodic2, g);
            for (int a = 0; a < 4; ++a)
                for (int d = 0; d < 3; ++d) x[a][d] = xyz[g[a] * 3 + d];
            double sd = element_matrix(kind, x, kind == 1 ? coef + cell * 3 : NULL,
                                       kind == 2 ? coef[tet] : 0.0, d_iso, d_ani, nu, t,
                                       Ke + tet * ne * ne);
            orient[tet] = sd > 0.0 ? 1 : (sd < 0.0 ? -1 : 0);
        }
    }
    /* every tet must be non-degenerate and oriented like the first one */
    for (int64_t tet = 0; tet < ntets; ++tet)
        if (orient[tet] == 0 || orient[tet] != orient[0]) {
            *bad_tet = tet;
            free(deg); free(adj); free(Ke); free(orient);
            return -3;
        }

    /* 2. CSR pattern: row (dpn*a + c) holds columns dpn*b + d for b in adj(a) */
    rowptr[0] = 0;
    for (int64_t a = 0; a < nn; ++a)
        for (int c = 0; c < dpn; ++c) {
            int64_t r = a * dpn + c;
            rowptr[r + 1] = rowptr[r] + (int64_t)deg[a] * dpn;
        }
    int32_t* gridof = (int32_t*)malloc((size_t)nn * sizeof(int32_t));
    if (!gridof) { free(deg); free(adj); free(Ke); free(orient); return -2; }
    for (int64_t g = 0; g < nn; ++g) gridof[newid[g]] = (int32_t)g;

    /* 3. rows in parallel: sum the incident tets' contributions in ascending tet order */
#pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < nn; ++a) {
        for (int c = 0; c < dpn; ++c) {
            int64_t p = rowptr[a * dpn + c];
            for (int k = 0; k < deg[a]; ++k)
                for (int d = 0; d < dpn; ++d) {
                    colind[p] = adj[a * FEGEN_MAX_DEG + k] * dpn + d;
                    values[p] = 0.0;
                    ++p;
                }
        }
        int64_t g = gridof[a];
        int i0 = (int)(g / ((int64_t)n1 * n2)), i1 = (int)((g / n2) % n1), i2 = (int)(g % n2);
        int64_t tets[48];
        int lv[48];
        int nt = 0;
        for (int d0 = 0; d0 < 2; ++d0)
            for (int d1 = 0; d1 < 2; ++d1)
                for (int d2 = 0; d2 < 2; ++d2) {
                    int c0 = i0 - d0, c1 = i1 - d1, c2 = i2 - d2;
                    if (c0 < 0 || c0 >= n0 - 1 || c1 < 0 || c1 >= n1 - 1) continue;
                    if (periodic2) {
                        c2 = (c2 + n2) % n2;
                    } else if (c2 < 0 || c2 >= n2 - 1) {
                        continue;
                    }
                    int64_t cell = ((int64_t)c0 * (n1 - 1) + c1) * nc2 + c2;
                    for (int t = 0; t < 6; ++t) {
                        int k = local_vertex(c0, c1, c2, t, n1, n2, periodic2, g);
                        if (k >= 0) { tets[nt] = cell * 6 + t; lv[nt] = k; ++nt; }
                    }
                }
        for (int i = 1; i < nt; ++i) {     /* ascending tet id */
            int64_t v = tets[i];
            int l = lv[i], j = i - 1;
            while (j >= 0 && tets[j] > v) { tets[j + 1] = tets[j]; lv[j + 1] = lv[j]; --j; }
            tets[j + 1] = v;
            lv[j + 1] = l;
        }
        const int32_t* row = adj + a * FEGEN_MAX_DEG;
        for (int q = 0; q < nt; ++q) {
            int64_t tet = tets[q];
            int64_t cell = tet / 6;
            int t = (int)(tet % 6);
            int c0 = (int)(cell / ((int64_t)(n1 - 1) * nc2));
            int c1 = (int)((cell / nc2) % (n1 - 1));
            int c2 = (int)(cell % nc2);
            int64_t vg[4];
            tet_nodes(c0, c1, c2, t, n1, n2, periodic2, vg);
            const double* K = Ke + tet * ne * ne;
            int la = lv[q];
            for (int b = 0; b < 4; ++b) {
                int32_t kcol = find_col(row, deg[a], newid[vg[b]]);
                for (int ci = 0; ci < dpn; ++ci) {
                    int64_t base = rowptr[a * dpn + ci] + (int64_t)kcol * dpn;
                    for (int cj = 0; cj < dpn; ++cj)
                        values[base + cj] += K[(dpn * la + ci) * ne + dpn * b + cj];
                }
            }
        }
    }
    free(gridof);
    free(deg);
    free(adj);
    free(Ke);
    free(orient);
    return 0;
}

/*
 * The element quantities behind fegen_assemble, in the same tet order (cell
 * major, 6 tets per cell): each tet's 4 node numbers (new numbering) in
 * elem_nodes[4 * tet + a], and its element matrix (ne x ne, ne = 4 * dofs per
 * node, row/column dpn * a + c for component c of vertex a) in
 * Ke[tet * ne * ne ...].  Returns 0, or -3 with *bad_tet for a degenerate tet.
 */
int fegen_elements(int kind, int n0, int n1, int n2, int periodic2, const double* xyz,
                   const int32_t* newid, const double* coef, double d_iso, double d_ani,
                   double nu, int32_t* elem_nodes, double* Ke, int64_t* bad_tet) {
    int dpn = (kind == 2) ? 3 : 1;
    int ne = 4 * dpn;
    int64_t nc2 = n_cells2(n2, periodic2);
    int64_t ncells = (int64_t)(n0 - 1) * (n1 - 1) * nc2;
    int64_t bad = -1;
#pragma omp parallel for schedule(static)
    for (int64_t cell = 0; cell < ncells; ++cell) {
        int c0 = (int)(cell / ((int64_t)(n1 - 1) * nc2));
        int c1 = (int)((cell / nc2) % (n1 - 1));
        int c2 = (int)(cell % nc2);
        for (int t = 0; t < 6; ++t) {
            int64_t tet = cell * 6 + t;
            int64_t g[4];
            double x[4][3];
            tet_nodes(c0, c1, c2, t, n1, n2, periodic2, g);
            for (int a = 0; a < 4; ++a) {
                elem_nodes[tet * 4 + a] = newid[g[a]];
                for (int d = 0; d < 3; ++d) x[a][d] = xyz[g[a] * 3 + d];
            }
            double sd = element_matrix(kind, x, kind == 1 ? coef + cell * 3 : NULL,
                                       kind == 2 ? coef[tet] : 0.0, d_iso, d_ani, nu, t,
                                       Ke + tet * ne * ne);
            if (sd == 0.0) {
#pragma omp critical
                bad = tet;
            }
        }
    }
    if (bad >= 0) { *bad_tet = bad; return -3; }
    return 0;
}

/*
 * Homogeneous Dirichlet conditions by symmetric elimination: every row r with
 * mask[r] != 0 becomes the identity row; every entry (i, j) with exactly one of
 * i, j constrained is dropped from the pattern.  Compacts the CSR in place and
 * returns the new nnz.
 */
int64_t fegen_dirichlet(int64_t n_rows, int64_t* rowptr, int32_t* colind, double* values,
                        const uint8_t* mask) {
    int64_t w = 0;
    int64_t start = rowptr[0];
    for (int64_t r = 0; r < n_rows; ++r) {
        int64_t end = rowptr[r + 1];
        int64_t new_start = w;
        for (int64_t p = start; p < end; ++p) {
            int32_t c = colind[p];
            if (mask[r]) {
                if (c == r) { colind[w] = c; values[w] = 1.0; ++w; }
            } else if (!mask[c]) {
                colind[w] = c; values[w] = values[p]; ++w;
            }
        }
        start = end;
        rowptr[r] = new_start;
    }
    rowptr[n_rows] = w;
    return w;
}
