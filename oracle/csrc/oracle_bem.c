/*
 * Oracle (test infrastructure only): plain FP64 dense collocation BEM rows.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
 * load this library. It shares no code with the CUDA path.
 *
 * Each routine follows the paper's mat-vec loop (Appendix, Algorithm
 * "Matrix-vector multiplication"): for every collocation point i, for every
 * integration panel j, add v_j times the integral of the kernel over panel j.
 * The integral over panel j is taken by one of three regimes (Sec. 2.3):
 *   - j == i            : the singular self-integral, done semi-analytically
 *                         (Hess-Smith polar decomposition, radial part in
 *                         closed form; the angular part is also closed form
 *                         for a flat panel);
 *   - |c_i - c_j| < f*sqrt(2 S_j), f = 2 by default : the near-singular rule
 *                         (K ~ 20 points);
 *   - otherwise          : the far rule with K points, eq. gauss:1st-kind /
 *                         gauss:2nd-kind: sum_k q_k S_j K(x_i, x_k).
 * Collocation points are panel centroids. Quadrature rules arrive as
 * barycentric coordinates plus area-normalised weights (sum q_k = 1).
 *
 * Operators (G = 1/(4 pi r), eq. laplace_bem_final; Stokeslet eq. stokeslet;
 * stresslet eq. stresslet):
 *   Laplace SL : V_ij = 1/(4 pi) int_j 1/|c_i - y| dS_y
 *   Laplace DL : K_ij = 1/(4 pi) int_j n_j . (c_i - y)/|c_i - y|^3 dS_y   (self = 0)
 *   Stokes SL  : A_iJ = -1/(8 pi mu) int_J [ I/r + d d^T/r^3 ] dS_y, d = c_i - y
 *   Stokes DL  : B_iJ[a][b] = 1/(8 pi) int_J 6 e_a e_b (e . n_J)/r^5 dS_y,
 *                e = y - c_i (the paper's T_ijk with x the integration point) (self = 0)
 * Rows are evaluated for the listed row indices; y_r = sum_j A_{row_r, j} x_j.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define PI 3.14159265358979323846

typedef struct {
    double c[3], n[3], S;
    double v[3][3];
} panel_t;

static void make_panel(const double *v9, panel_t *P) {
    double e1[3], e2[3], cr[3];
    for (int a = 0; a < 3; ++a) {
        for (int d = 0; d < 3; ++d) P->v[a][d] = v9[3 * a + d];
    }
    for (int d = 0; d < 3; ++d) {
        P->c[d] = (P->v[0][d] + P->v[1][d] + P->v[2][d]) / 3.0;
        e1[d] = P->v[1][d] - P->v[0][d];
        e2[d] = P->v[2][d] - P->v[0][d];
    }
    cr[0] = e1[1] * e2[2] - e1[2] * e2[1];
    cr[1] = e1[2] * e2[0] - e1[0] * e2[2];
    cr[2] = e1[0] * e2[1] - e1[1] * e2[0];
    double len = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    for (int d = 0; d < 3; ++d) P->n[d] = cr[d] / len;
    P->S = 0.5 * len;
}

static void bary_point(const panel_t *P, const double *l, double y[3]) {
    for (int d = 0; d < 3; ++d) y[d] = l[0] * P->v[0][d] + l[1] * P->v[1][d] + l[2] * P->v[2][d];
}

/* Integral over the flat panel of 1/|c - y| and of d d^T/|d|^3 (d = c - y),
 * for a point c inside the panel and in its plane. The panel is split into
 * the three triangles (c, P_a, P_b) over its edges; in polar coordinates
 * about c the radial integral is exact and, for a straight edge at distance
 * h, the angular integral is elementary:
 *   int 1/r dA                = h [asinh(s/h)]_{s1}^{s2}
 *   int e e^T (h/cos psi) dpsi = h { [sin psi] u u^T - [cos psi] (u v^T + v u^T)
 *                                    + [asinh(tan psi) - sin psi] v v^T }
 * with u the unit vector from c to the foot of the perpendicular on the edge,
 * v the edge direction, tan psi = s/h. */
void oracle_self_integrals(const double *v9, const double *c, double *inv_r, double *ddT) {
    panel_t P;
    make_panel(v9, &P);
    double I1 = 0.0, D[3][3] = {{0}};
    for (int a = 0; a < 3; ++a) {
        const double *A = P.v[a], *B = P.v[(a + 1) % 3];
        double e[3], L = 0.0, t = 0.0;
        for (int d = 0; d < 3; ++d) { e[d] = B[d] - A[d]; L += e[d] * e[d]; }
        L = sqrt(L);
        for (int d = 0; d < 3; ++d) e[d] /= L;
        for (int d = 0; d < 3; ++d) t += (c[d] - A[d]) * e[d];
        double F[3], u[3], h = 0.0;
        for (int d = 0; d < 3; ++d) { F[d] = A[d] + t * e[d]; u[d] = F[d] - c[d]; h += u[d] * u[d]; }
        h = sqrt(h);
        for (int d = 0; d < 3; ++d) u[d] /= h;
        double s1 = -t, s2 = L - t;
        double r1 = sqrt(s1 * s1 + h * h), r2 = sqrt(s2 * s2 + h * h);
        double as = asinh(s2 / h) - asinh(s1 / h);
        I1 += h * as;
        double dsin = s2 / r2 - s1 / r1;
        double dcos = h / r2 - h / r1;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                D[i][j] += h * (dsin * u[i] * u[j] - dcos * (u[i] * e[j] + e[i] * u[j]) + (as - dsin) * e[i] * e[j]);
    }
    *inv_r = I1;
    if (ddT) for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) ddT[3 * i + j] = D[i][j];
}

typedef struct {
    int n;
    const double *verts;      /* n x 9: the three vertices of each panel */
    int kf; const double *fb, *fw;   /* far rule: kf x 3 barycentric, kf weights */
    int kn; const double *nb, *nw;   /* near rule */
    double near_factor;
} mesh_t;

static int is_near(const panel_t *Pi, const panel_t *Pj, double f) {
    double d2 = 0.0;
    for (int d = 0; d < 3; ++d) { double t = Pi->c[d] - Pj->c[d]; d2 += t * t; }
    double R = f * sqrt(2.0 * Pj->S);
    return d2 < R * R;
}

/* Laplace row entries for target panel i. kind 0 = SL, 1 = DL. Unscaled (no 1/(4 pi)). */
static double laplace_entry(const mesh_t *M, const panel_t *Pi, int i, const panel_t *Pj, int j, int kind) {
    if (i == j) {
        if (kind == 1) return 0.0;
        double I1;
        oracle_self_integrals(M->verts + 9 * (size_t)j, Pi->c, &I1, 0);
        return I1;
    }
    int near = is_near(Pi, Pj, M->near_factor);
    int K = near ? M->kn : M->kf;
    const double *b = near ? M->nb : M->fb, *w = near ? M->nw : M->fw;
    double s = 0.0;
    for (int k = 0; k < K; ++k) {
        double y[3], d[3];
        bary_point(Pj, b + 3 * k, y);
        for (int a = 0; a < 3; ++a) d[a] = Pi->c[a] - y[a];
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        if (kind == 0) s += w[k] * Pj->S / r;
        else s += w[k] * Pj->S * (Pj->n[0] * d[0] + Pj->n[1] * d[1] + Pj->n[2] * d[2]) / (r * r * r);
    }
    return s;
}

/* y[r] = sum_j A[rows[r], j] x[j]; if Aout != NULL also stores the rows (nrows x n). */
void oracle_laplace_rows(int n, const double *verts, int kf, const double *fb, const double *fw,
                         int kn, const double *nb, const double *nw, double near_factor, int kind,
                         int nrows, const int64_t *rows, const double *x, double *y, double *Aout) {
    mesh_t M = {n, verts, kf, fb, fw, kn, nb, nw, near_factor};
    const double scale = 1.0 / (4.0 * PI);
#pragma omp parallel for schedule(dynamic, 4)
    for (int r = 0; r < nrows; ++r) {
        int i = (int)rows[r];
        panel_t Pi, Pj;
        make_panel(verts + 9 * (size_t)i, &Pi);
        double acc = 0.0;
        for (int j = 0; j < n; ++j) {
            make_panel(verts + 9 * (size_t)j, &Pj);
            double a = scale * laplace_entry(&M, &Pi, i, &Pj, j, kind);
            if (x) acc += a * x[j];
            if (Aout) Aout[(size_t)r * n + j] = a;
        }
        if (y) y[r] = acc;
    }
}

/* Stokes 3x3 block for target i, source panel J. kind 0 = Stokeslet SL (unscaled
 * int G dS), kind 1 = stresslet DL (unscaled int T_abk n_k dS). */
static void stokes_block(const mesh_t *M, const panel_t *Pi, int i, const panel_t *Pj, int j, int kind, double B[9]) {
    memset(B, 0, 9 * sizeof(double));
    if (i == j) {
        if (kind == 1) return;
        double I1, D[9];
        oracle_self_integrals(M->verts + 9 * (size_t)j, Pi->c, &I1, D);
        for (int a = 0; a < 9; ++a) B[a] = D[a];
        B[0] += I1; B[4] += I1; B[8] += I1;
        return;
    }
    int near = is_near(Pi, Pj, M->near_factor);
    int K = near ? M->kn : M->kf;
    const double *b = near ? M->nb : M->fb, *w = near ? M->nw : M->fw;
    for (int k = 0; k < K; ++k) {
        double y[3], d[3];
        bary_point(Pj, b + 3 * k, y);
        for (int a = 0; a < 3; ++a) d[a] = Pi->c[a] - y[a];
        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2], r = sqrt(r2);
        double wq = w[k] * Pj->S;
        if (kind == 0) {
            for (int a = 0; a < 3; ++a)
                for (int c = 0; c < 3; ++c)
                    B[3 * a + c] += wq * ((a == c ? 1.0 / r : 0.0) + d[a] * d[c] / (r2 * r));
        } else {
            /* e = y - c_i = -d; T_abk n_k = 6 e_a e_b (e.n) / r^5 */
            double en = -(d[0] * Pj->n[0] + d[1] * Pj->n[1] + d[2] * Pj->n[2]);
            double r5 = r2 * r2 * r;
            for (int a = 0; a < 3; ++a)
                for (int c = 0; c < 3; ++c)
                    B[3 * a + c] += wq * 6.0 * d[a] * d[c] * en / r5;
        }
    }
}

/* Stokes rows: unknowns are 3 per panel (x[3j+c]); rows[r] indexes panels; the
 * output y has 3 entries per listed panel. Aout (optional) is (3 nrows) x (3 n). */
void oracle_stokes_rows(int n, const double *verts, int kf, const double *fb, const double *fw,
                        int kn, const double *nb, const double *nw, double near_factor, int kind, double mu,
                        int nrows, const int64_t *rows, const double *x, double *y, double *Aout) {
    mesh_t M = {n, verts, kf, fb, fw, kn, nb, nw, near_factor};
    const double scale = (kind == 0) ? -1.0 / (8.0 * PI * mu) : 1.0 / (8.0 * PI);
#pragma omp parallel for schedule(dynamic, 4)
    for (int r = 0; r < nrows; ++r) {
        int i = (int)rows[r];
        panel_t Pi, Pj;
        make_panel(verts + 9 * (size_t)i, &Pi);
        double acc[3] = {0, 0, 0}, B[9];
        for (int j = 0; j < n; ++j) {
            make_panel(verts + 9 * (size_t)j, &Pj);
            stokes_block(&M, &Pi, i, &Pj, j, kind, B);
            for (int a = 0; a < 3; ++a) {
                for (int c = 0; c < 3; ++c) {
                    double e = scale * B[3 * a + c];
                    if (x) acc[a] += e * x[3 * j + c];
                    if (Aout) Aout[(size_t)(3 * r + a) * (3 * (size_t)n) + 3 * j + c] = e;
                }
            }
        }
        if (y) for (int a = 0; a < 3; ++a) y[3 * r + a] = acc[a];
    }
}

/* Plain N-body sums (the FMM's target, eq. nbody): phi_i = sum_j q_j / |x_i - y_j|,
 * and grad_i = sum_j q_j * -(x_i - y_j)/|x_i - y_j|^3 when grad != NULL. */
void oracle_nbody_laplace(int nt, const double *tx, int ns, const double *sy, const double *q,
                          double *phi, double *grad) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < nt; ++i) {
        double p = 0.0, g[3] = {0, 0, 0};
        for (int j = 0; j < ns; ++j) {
            double d[3] = {tx[3 * i] - sy[3 * j], tx[3 * i + 1] - sy[3 * j + 1], tx[3 * i + 2] - sy[3 * j + 2]};
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 == 0.0) continue;
            double r = sqrt(r2);
            p += q[j] / r;
            for (int a = 0; a < 3; ++a) g[a] -= q[j] * d[a] / (r2 * r);
        }
        phi[i] = p;
        if (grad) for (int a = 0; a < 3; ++a) grad[3 * i + a] = g[a];
    }
}
