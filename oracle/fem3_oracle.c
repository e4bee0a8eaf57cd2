/*
 * fem3_oracle.c - plain, slow FP64 CPU restatement of the fractional FEM assembly.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark may load this library.  It shares no code, header or constant
 * generator with the CUDA library; both sides read the same seeded inputs and
 * nothing else.
 *
 * What it computes (Yang, Nie, Yuan, Wang, "Finite Element Methods for Fractional
 * PDEs in Three Dimensions"):
 *   - Section 2.2: volume coordinates of a simplex, the ray-simplex intersection
 *     interval (the conditions b~ + r d~ >= 0, r >= 0) and the walk across the
 *     triangulation through the exit m-face named by the zero pattern of the volume
 *     coordinate (Fig. "fig:vc").
 *   - Section 2.1: the left/right Riemann-Liouville derivative of a P1 basis function
 *     along the path, summed segment by segment.  The paper promises but does not
 *     print the closed form; the one used here follows from integrating eq. "def" by
 *     parts on each segment where the basis function is linear:
 *        D_L^g phi(x) = phi(a) (x-a)^(-g)/Gamma(1-g)
 *                       + sum_k slope_k ((x-y0_k)^(1-g) - (x-y1_k)^(1-g)) / Gamma(2-g)
 *     (and the mirror image for D_R with a leading minus on the sum).  phi(a) = 0 for
 *     every interior basis function.
 *   - Section 2.1: element-sum Galerkin matrix with Gauss quadrature,
 *        A_jk = sum_i s_i K_i sum_g w_g (D_R phi_j D_L phi_k + D_L phi_j D_R phi_k)(x_g)
 *     with the Riesz constant s_i = 1/(2 cos(pi alpha_i/2)) and order g_i = alpha_i/2.
 *   - Section 2.1, eq. "equ:varsss": one axis term of the general form
 *     (c D^alpha u, D^^beta v) with a coefficient and unequal orders in [0, 1], and
 *     Section 3, eq. "equ:sfde2": the divergence-form operator with coefficients p_i, q_i
 *     through its variational form (not symmetric).
 *   - The dense SPD solve (textbook Cholesky), the P1 load vector and the adjoint.
 *
 * Parity of each function is pinned by tests against closed forms, brute force and
 * invariants (see tests/test_oracle_*.py); nothing here is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_E_ARG (-1)
#define OR_E_MESH (-2)
#define OR_E_WALK (-3)
#define OR_E_NOT_SPD (-4)
#define OR_E_OOM (-7)

/* Tolerances of the walk (the paper tests for exact zeros; floating point needs a
 * threshold).  Relative to O(1) volume coordinates, to the mesh span and to the
 * largest gradient component of the tetrahedron along the axis. */
static const double EPS_LAMBDA = 1e-12;
static const double EPS_R_REL = 1e-12;
static const double EPS_D_REL = 1e-12;

typedef struct {
    int64_t n_nodes, n_tets, n_dof, n_gp;
    double *verts;   /* [n_nodes][3] */
    int32_t *tets;   /* [n_tets][4] */
    double *M;       /* [n_tets][4][4]; row k: lambda_k(x) = M0 + M1 x + M2 y + M3 z */
    double *vol;     /* [n_tets] */
    int32_t *nbr;    /* [n_tets][4]: tet across the face opposite local vertex k, or -1 */
    int32_t *dof;    /* [n_nodes]: dof index (interior vertex) or -1 */
    int64_t *vt_off; /* [n_nodes+1] vertex -> tets CSR */
    int32_t *vt_tet;
    double *gp;      /* [4 n_tets][3] Gauss points */
    double *gw;      /* [4 n_tets] weights */
    double span;     /* largest extent of the bounding box */
    int max_steps;
} or_mesh;

/* 4-point degree-2 rule on a tetrahedron: barycentric permutations of (a,b,b,b). */
static double rule_a(void) { return (5.0 + 3.0 * sqrt(5.0)) / 20.0; }
static double rule_b(void) { return (5.0 - sqrt(5.0)) / 20.0; }

void or_mesh_free(or_mesh *m)
{
    if (!m) return;
    free(m->verts); free(m->tets); free(m->M); free(m->vol); free(m->nbr); free(m->dof);
    free(m->vt_off); free(m->vt_tet); free(m->gp); free(m->gw);
    free(m);
}

/* Inverse of the 4x4 matrix P = [[1,1,1,1],[v0 v1 v2 v3]] (columns [1; v_k]) by
 * Gauss-Jordan elimination with partial pivoting: lambda = P^{-1} [1; x]. */
static int inverse4(const double P[4][4], double Minv[4][4])
{
    double a[4][8];
    for (int r = 0; r < 4; r++)
        for (int c = 0; c < 8; c++)
            a[r][c] = c < 4 ? P[r][c] : (c - 4 == r ? 1.0 : 0.0);
    for (int c = 0; c < 4; c++) {
        int piv = c;
        for (int r = c + 1; r < 4; r++)
            if (fabs(a[r][c]) > fabs(a[piv][c])) piv = r;
        if (a[piv][c] == 0.0) return OR_E_MESH;
        if (piv != c)
            for (int k = 0; k < 8; k++) { double t = a[c][k]; a[c][k] = a[piv][k]; a[piv][k] = t; }
        double d = a[c][c];
        for (int k = 0; k < 8; k++) a[c][k] /= d;
        for (int r = 0; r < 4; r++) {
            if (r == c) continue;
            double f = a[r][c];
            for (int k = 0; k < 8; k++) a[r][k] -= f * a[c][k];
        }
    }
    for (int r = 0; r < 4; r++)
        for (int c = 0; c < 4; c++) Minv[r][c] = a[r][c + 4];
    return OR_OK;
}

typedef struct { int32_t v[3]; int32_t tet, k; } face_rec;

static int face_cmp(const void *pa, const void *pb)
{
    const face_rec *a = pa, *b = pb;
    for (int i = 0; i < 3; i++) {
        if (a->v[i] < b->v[i]) return -1;
        if (a->v[i] > b->v[i]) return 1;
    }
    if (a->tet != b->tet) return a->tet < b->tet ? -1 : 1;
    return a->k - b->k;
}

/* Build the mesh records: barycentric maps, volumes, face neighbours, boundary
 * vertices and dof numbering (interior vertices in ascending node order), the
 * vertex -> tet table, and the Gauss points.  Returns NULL on bad input and sets
 * *status. */
or_mesh *or_mesh_build(const double *verts, int64_t n_nodes, const int32_t *tets,
                       int64_t n_tets, int *status)
{
    *status = OR_E_ARG;
    if (!verts || !tets || n_nodes < 4 || n_tets < 1) return NULL;
    or_mesh *m = calloc(1, sizeof(or_mesh));
    if (!m) { *status = OR_E_OOM; return NULL; }
    m->n_nodes = n_nodes; m->n_tets = n_tets; m->n_gp = 4 * n_tets;
    m->verts = malloc(sizeof(double) * 3 * n_nodes);
    m->tets = malloc(sizeof(int32_t) * 4 * n_tets);
    m->M = malloc(sizeof(double) * 16 * n_tets);
    m->vol = malloc(sizeof(double) * n_tets);
    m->nbr = malloc(sizeof(int32_t) * 4 * n_tets);
    m->dof = malloc(sizeof(int32_t) * n_nodes);
    m->vt_off = calloc(n_nodes + 1, sizeof(int64_t));
    m->vt_tet = malloc(sizeof(int32_t) * 4 * n_tets);
    m->gp = malloc(sizeof(double) * 3 * m->n_gp);
    m->gw = malloc(sizeof(double) * m->n_gp);
    if (!m->verts || !m->tets || !m->M || !m->vol || !m->nbr || !m->dof || !m->vt_off ||
        !m->vt_tet || !m->gp || !m->gw) { or_mesh_free(m); *status = OR_E_OOM; return NULL; }
    memcpy(m->verts, verts, sizeof(double) * 3 * n_nodes);
    memcpy(m->tets, tets, sizeof(int32_t) * 4 * n_tets);

    /* span of the bounding box */
    double lo[3], hi[3];
    for (int d = 0; d < 3; d++) { lo[d] = verts[d]; hi[d] = verts[d]; }
    for (int64_t v = 0; v < n_nodes; v++)
        for (int d = 0; d < 3; d++) {
            if (verts[3 * v + d] < lo[d]) lo[d] = verts[3 * v + d];
            if (verts[3 * v + d] > hi[d]) hi[d] = verts[3 * v + d];
        }
    m->span = 0.0;
    for (int d = 0; d < 3; d++) if (hi[d] - lo[d] > m->span) m->span = hi[d] - lo[d];

    /* per tet: barycentric map and volume */
    for (int64_t t = 0; t < n_tets; t++) {
        double P[4][4];
        for (int k = 0; k < 4; k++) {
            int32_t v = tets[4 * t + k];
            if (v < 0 || v >= n_nodes) { or_mesh_free(m); *status = OR_E_MESH; return NULL; }
            P[0][k] = 1.0;
            for (int d = 0; d < 3; d++) P[1 + d][k] = verts[3 * v + d];
        }
        double e[3][3];
        for (int c = 0; c < 3; c++)
            for (int d = 0; d < 3; d++) e[c][d] = P[1 + d][c + 1] - P[1 + d][0];
        double det = e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1])
                   - e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0])
                   + e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
        m->vol[t] = fabs(det) / 6.0;
        if (!(m->vol[t] > 0.0)) { or_mesh_free(m); *status = OR_E_MESH; return NULL; }
        double Mi[4][4];
        if (inverse4(P, Mi) != OR_OK) { or_mesh_free(m); *status = OR_E_MESH; return NULL; }
        for (int k = 0; k < 4; k++)
            for (int c = 0; c < 4; c++) m->M[16 * t + 4 * k + c] = Mi[k][c];
    }

    /* face neighbours by sorting face keys */
    face_rec *fr = malloc(sizeof(face_rec) * 4 * n_tets);
    if (!fr) { or_mesh_free(m); *status = OR_E_OOM; return NULL; }
    for (int64_t t = 0; t < n_tets; t++)
        for (int k = 0; k < 4; k++) {
            face_rec *f = &fr[4 * t + k];
            int n = 0;
            for (int q = 0; q < 4; q++) if (q != k) f->v[n++] = tets[4 * t + q];
            /* sort the three vertex ids */
            for (int a = 0; a < 3; a++)
                for (int b = a + 1; b < 3; b++)
                    if (f->v[b] < f->v[a]) { int32_t s = f->v[a]; f->v[a] = f->v[b]; f->v[b] = s; }
            f->tet = (int32_t)t; f->k = k;
        }
    qsort(fr, 4 * n_tets, sizeof(face_rec), face_cmp);
    for (int64_t i = 0; i < 4 * n_tets; i++) m->nbr[4 * fr[i].tet + fr[i].k] = -1;
    for (int64_t i = 0; i < 4 * n_tets;) {
        int64_t j = i + 1;
        while (j < 4 * n_tets && fr[j].v[0] == fr[i].v[0] && fr[j].v[1] == fr[i].v[1] &&
               fr[j].v[2] == fr[i].v[2]) j++;
        if (j - i > 2) { free(fr); or_mesh_free(m); *status = OR_E_MESH; return NULL; }
        if (j - i == 2) {
            m->nbr[4 * fr[i].tet + fr[i].k] = fr[i + 1].tet;
            m->nbr[4 * fr[i + 1].tet + fr[i + 1].k] = fr[i].tet;
        }
        i = j;
    }
    free(fr);

    /* boundary vertices: those on a face without neighbour; unused nodes are not dofs */
    char *bnd = calloc(n_nodes, 1), *used = calloc(n_nodes, 1);
    if (!bnd || !used) { free(bnd); free(used); or_mesh_free(m); *status = OR_E_OOM; return NULL; }
    for (int64_t t = 0; t < n_tets; t++)
        for (int k = 0; k < 4; k++) {
            used[tets[4 * t + k]] = 1;
            if (m->nbr[4 * t + k] < 0)
                for (int q = 0; q < 4; q++) if (q != k) bnd[tets[4 * t + q]] = 1;
        }
    m->n_dof = 0;
    for (int64_t v = 0; v < n_nodes; v++)
        m->dof[v] = (used[v] && !bnd[v]) ? (int32_t)(m->n_dof++) : -1;
    free(bnd); free(used);

    /* vertex -> tets, tets in increasing order */
    for (int64_t t = 0; t < n_tets; t++)
        for (int k = 0; k < 4; k++) m->vt_off[tets[4 * t + k] + 1]++;
    for (int64_t v = 0; v < n_nodes; v++) m->vt_off[v + 1] += m->vt_off[v];
    int64_t *cur = malloc(sizeof(int64_t) * n_nodes);
    if (!cur) { or_mesh_free(m); *status = OR_E_OOM; return NULL; }
    memcpy(cur, m->vt_off, sizeof(int64_t) * n_nodes);
    for (int64_t t = 0; t < n_tets; t++)
        for (int k = 0; k < 4; k++) m->vt_tet[cur[tets[4 * t + k]]++] = (int32_t)t;
    free(cur);

    /* Gauss points: point q of tet t has barycentric a at vertex q and b elsewhere */
    double a = rule_a(), b = rule_b();
    for (int64_t t = 0; t < n_tets; t++)
        for (int q = 0; q < 4; q++) {
            int64_t g = 4 * t + q;
            for (int d = 0; d < 3; d++) {
                double x = 0.0;
                for (int k = 0; k < 4; k++)
                    x += (k == q ? a : b) * verts[3 * tets[4 * t + k] + d];
                m->gp[3 * g + d] = x;
            }
            m->gw[g] = m->vol[t] / 4.0;
        }
    m->max_steps = (int)(8.0 * cbrt((double)n_tets)) + 64;
    *status = OR_OK;
    return m;
}

void or_mesh_info(const or_mesh *m, int64_t *n_dof, int64_t *n_gp, double *span)
{
    *n_dof = m->n_dof; *n_gp = m->n_gp; *span = m->span;
}

/* Copy the records out (any pointer may be NULL). */
void or_mesh_get(const or_mesh *m, double *M, double *vol, int32_t *nbr, int32_t *dof,
                 double *gp, double *gw)
{
    if (M) memcpy(M, m->M, sizeof(double) * 16 * m->n_tets);
    if (vol) memcpy(vol, m->vol, sizeof(double) * m->n_tets);
    if (nbr) memcpy(nbr, m->nbr, sizeof(int32_t) * 4 * m->n_tets);
    if (dof) memcpy(dof, m->dof, sizeof(int32_t) * m->n_nodes);
    if (gp) memcpy(gp, m->gp, sizeof(double) * 3 * m->n_gp);
    if (gw) memcpy(gw, m->gw, sizeof(double) * m->n_gp);
}

/* Volume coordinates of the ray start x in tet t (b~ of Section 2.2) and the direction
 * d~ = dir * (column 1+axis of the barycentric map). */
static void ray_in_tet(const or_mesh *m, int32_t t, const double *x, int axis, int dir,
                       double bt[4], double dt[4], double *dscale)
{
    const double *M = m->M + 16 * (int64_t)t;
    *dscale = 0.0;
    for (int k = 0; k < 4; k++) {
        bt[k] = M[4 * k] + M[4 * k + 1] * x[0] + M[4 * k + 2] * x[1] + M[4 * k + 3] * x[2];
        dt[k] = dir * M[4 * k + 1 + axis];
        if (fabs(dt[k]) > *dscale) *dscale = fabs(dt[k]);
    }
}

/* Largest r with b~ + r d~ >= 0 (the go-out parameter r_max of the intersection
 * interval).  Components with d~_k >= 0 (up to the tolerance) never bound it. */
static double interval_rmax(const double bt[4], const double dt[4], double dscale)
{
    double rmax = INFINITY;
    for (int k = 0; k < 4; k++)
        if (dt[k] < -EPS_D_REL * dscale) {
            double r = -bt[k] / dt[k];
            if (r < rmax) rmax = r;
        }
    return rmax;
}

/* Walk the ray x + r * dir * e_axis, r >= 0, from tet t0 (which must hold x) to the
 * boundary.  Segments (tet, r_in, r_out) are written in order; their lengths
 * telescope to r_end, the distance from x to a_axis(x) (dir = -1) or b_axis(x)
 * (dir = +1).  Returns the number of segments, or a negative error. */
int or_walk_point(const or_mesh *m, const double *x, int32_t t0, int axis, int dir, int cap,
                  int32_t *seg_tet, double *seg_r0, double *seg_r1, double *r_end_out,
                  int32_t *end_tet_out)
{
    if (t0 < 0 || t0 >= m->n_tets || axis < 0 || axis > 2 || (dir != 1 && dir != -1))
        return OR_E_ARG;
    const double eps_r = EPS_R_REL * m->span;
    int32_t t = t0;
    double r_prev = 0.0;
    int nseg = 0;
    for (int step = 0; step < m->max_steps; step++) {
        double bt[4], dt[4], ds;
        ray_in_tet(m, t, x, axis, dir, bt, dt, &ds);
        double rmax = interval_rmax(bt, dt, ds);
        if (!(rmax < INFINITY)) return OR_E_WALK;
        if (rmax - r_prev > eps_r) {
            /* a segment of positive length (Section 2.2: an empty or one-point
             * interval contributes nothing) */
            if (nseg >= cap) return OR_E_WALK;
            seg_tet[nseg] = t; seg_r0[nseg] = r_prev; seg_r1[nseg] = rmax;
            nseg++;
            r_prev = rmax;
        }
        /* zero pattern of the go-out volume coordinate names the exit m-face */
        int inZ[4], nz = 0;
        for (int k = 0; k < 4; k++) {
            double lam = bt[k] + rmax * dt[k];
            inZ[k] = lam <= EPS_LAMBDA;
            nz += inZ[k];
        }
        int32_t next = -1;
        if (nz == 1) {
            for (int k = 0; k < 4; k++) if (inZ[k]) next = m->nbr[4 * (int64_t)t + k];
        } else if (nz >= 2 && nz <= 3) {
            /* edge or vertex exit: search every tet holding the m-face (the vertices
             * of t outside the zero set); keep those the ray continues into, prefer the
             * longest continuation, then the smallest id */
            int32_t fv[4]; int nf = 0;
            for (int k = 0; k < 4; k++) if (!inZ[k]) fv[nf++] = m->tets[4 * (int64_t)t + k];
            int32_t v0 = fv[0];
            /* pass 1: longest continuation; pass 2: smallest id within eps_r of it */
            double best = -INFINITY;
            for (int pass = 0; pass < 2; pass++) {
                for (int64_t c = m->vt_off[v0]; c < m->vt_off[v0 + 1]; c++) {
                    int32_t u = m->vt_tet[c];
                    if (u == t) continue;
                    int has_all = 1;
                    for (int f = 1; f < nf; f++) {
                        int found = 0;
                        for (int q = 0; q < 4; q++) if (m->tets[4 * (int64_t)u + q] == fv[f]) found = 1;
                        has_all &= found;
                    }
                    if (!has_all) continue;
                    double bu[4], du[4], dsu;
                    ray_in_tet(m, u, x, axis, dir, bu, du, &dsu);
                    double ru = interval_rmax(bu, du, dsu);
                    if (!(ru > rmax + eps_r)) continue;
                    if (pass == 0) {
                        if (ru > best) best = ru;
                    } else if (ru >= best - eps_r && (next < 0 || u < next)) {
                        next = u;
                    }
                }
            }
        } else {
            return OR_E_WALK;
        }
        if (next < 0) {
            if (r_end_out) *r_end_out = r_prev;
            if (end_tet_out) *end_tet_out = t;
            return nseg;
        }
        t = next;
    }
    return OR_E_WALK;
}

/* The walk from Gauss point g (it lies inside tet g / 4). */
int or_walk(const or_mesh *m, int64_t g, int axis, int dir, int cap, int32_t *seg_tet,
            double *seg_r0, double *seg_r1, double *r_end_out, int32_t *end_tet_out)
{
    if (g < 0 || g >= m->n_gp) return OR_E_ARG;
    return or_walk_point(m, m->gp + 3 * g, (int32_t)(g / 4), axis, dir, cap, seg_tet, seg_r0,
                         seg_r1, r_end_out, end_tet_out);
}

/* One row of a derivative table: row[j] = D_L^gamma phi_j(x_g) (dir = -1) or
 * D_R^gamma phi_j(x_g) (dir = +1) along axis.  all_nodes = 0 fills the n_dof interior
 * basis functions (phi_j(a) = 0, no boundary term); all_nodes = 1 fills all n_nodes
 * basis functions and adds the boundary term phi_j(end) r_end^(-gamma)/Gamma(1-gamma). */
int or_table_row(const or_mesh *m, int64_t g, int axis, int dir, double gamma,
                 int all_nodes, double *row)
{
    int cap = m->max_steps;
    int32_t *st = malloc(sizeof(int32_t) * cap);
    double *r0 = malloc(sizeof(double) * cap), *r1 = malloc(sizeof(double) * cap);
    if (!st || !r0 || !r1) { free(st); free(r0); free(r1); return OR_E_OOM; }
    double r_end; int32_t t_end;
    int ns = or_walk(m, g, axis, dir, cap, st, r0, r1, &r_end, &t_end);
    if (ns < 0) { free(st); free(r0); free(r1); return ns; }
    int64_t len = all_nodes ? m->n_nodes : m->n_dof;
    memset(row, 0, sizeof(double) * len);
    double p = 1.0 - gamma, G2 = tgamma(2.0 - gamma);
    double sgn = dir < 0 ? 1.0 : -1.0;
    for (int s = 0; s < ns; s++) {
        double pf = pow(r1[s], p);
        double pn = r0[s] > 0.0 ? pow(r0[s], p) : 0.0;
        double coef = sgn * (pf - pn) / G2;
        const double *M = m->M + 16 * (int64_t)st[s];
        for (int v = 0; v < 4; v++) {
            int32_t node = m->tets[4 * (int64_t)st[s] + v];
            int64_t j = all_nodes ? node : m->dof[node];
            if (j >= 0) row[j] += coef * M[4 * v + 1 + axis];
        }
    }
    if (all_nodes && gamma < 1.0 && ns > 0) {
        double bt[4], dt[4], ds;
        ray_in_tet(m, t_end, m->gp + 3 * g, axis, dir, bt, dt, &ds);
        double scale = pow(r_end, -gamma) / tgamma(1.0 - gamma);
        for (int v = 0; v < 4; v++) {
            double lam = bt[v] + r_end * dt[v];
            row[m->tets[4 * (int64_t)t_end + v]] += lam * scale;
        }
    }
    free(st); free(r0); free(r1);
    return OR_OK;
}

/* Dense FP64 stiffness matrix, row-major [n_dof][n_dof]:
 *   A = sum_i s_i K_i sum_g w_g (R_i[g,:]^T L_i[g,:] + L_i[g,:]^T R_i[g,:])
 * with L_i = D_L^{alpha_i/2}, R_i = D_R^{alpha_i/2} tables.  Both products are added
 * separately (symmetry is a test, not a construction). */
int or_assemble(const or_mesh *m, const double alpha[3], const double K[3], double *A)
{
    int64_t n = m->n_dof;
    memset(A, 0, sizeof(double) * n * n);
    double *L = calloc(n > 0 ? n : 1, sizeof(double)), *R = calloc(n > 0 ? n : 1, sizeof(double));
    int64_t *iL = malloc(sizeof(int64_t) * (n > 0 ? n : 1)), *iR = malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    if (!L || !R || !iL || !iR) { free(L); free(R); free(iL); free(iR); return OR_E_OOM; }
    for (int axis = 0; axis < 3; axis++) {
        if (!(alpha[axis] > 1.0 && alpha[axis] <= 2.0)) { free(L); free(R); free(iL); free(iR); return OR_E_ARG; }
        double gamma = alpha[axis] / 2.0;
        double s = 1.0 / (2.0 * cos(M_PI * alpha[axis] / 2.0));
        double c = s * K[axis];
        for (int64_t g = 0; g < m->n_gp; g++) {
            int e1 = or_table_row(m, g, axis, -1, gamma, 0, L);
            int e2 = or_table_row(m, g, axis, +1, gamma, 0, R);
            if (e1 || e2) { free(L); free(R); free(iL); free(iR); return e1 ? e1 : e2; }
            int64_t nl = 0, nr = 0;
            for (int64_t j = 0; j < n; j++) {
                if (L[j] != 0.0) iL[nl++] = j;
                if (R[j] != 0.0) iR[nr++] = j;
            }
            double cw = c * m->gw[g];
            for (int64_t a = 0; a < nl; a++)
                for (int64_t b = 0; b < nr; b++)
                    A[iL[a] * n + iR[b]] += cw * L[iL[a]] * R[iR[b]];
            for (int64_t a = 0; a < nr; a++)
                for (int64_t b = 0; b < nl; b++)
                    A[iR[a] * n + iL[b]] += cw * R[iR[a]] * L[iL[b]];
        }
    }
    free(L); free(R); free(iL); free(iR);
    return OR_OK;
}

/* One axis term of the general bilinear form of Section 2.1, (c D^alpha u, D^^beta v)
 * (eq. "equ:varsss"), by the Gauss-quadrature element formula that follows it:
 *   K[k][l] = sum_g w_g c(x_g) (D^alpha psi_l)(x_g) (D^^beta psi_k)(x_g),
 * l the trial (column) and k the test (row) basis function.  D^alpha is the left
 * operator and D^^beta the right one when trial_left = 1, the other way round when 0.
 * Orders in [0, 1] (the tables of or_table_row: order 0 is the function itself, order 1
 * its first derivative, with a minus sign for the right operator).  c: [n_gp] values of
 * the coefficient at the Gauss points, or NULL for c = 1.  all_nodes = 1: rows and
 * columns over every node (tables with their boundary terms); 0: interior dofs.  K:
 * row-major [n][n].  The Riesz term of or_assemble is s K (form(L, R) + form(R, L)) at
 * alpha = beta = alpha_i / 2 and c = 1. */
/* The Section 2.1 element sum restricted to the listed Gauss points: adds, for every axis,
 * s_i K_i w_g (L[g] R[g]^T + R[g] L[g]^T) of each listed g to A (A is not cleared).  The
 * sum over a partition of all Gauss points is or_assemble's matrix (up to the order of
 * the floating-point additions).  Used to time the oracle on a bounded sample of lines. */
int or_assemble_gps(const or_mesh *m, const double alpha[3], const double K[3],
                    const int64_t *gps, int64_t n_g, double *A)
{
    int64_t n = m->n_dof;
    double *L = calloc(n > 0 ? n : 1, sizeof(double)), *R = calloc(n > 0 ? n : 1, sizeof(double));
    int64_t *iL = malloc(sizeof(int64_t) * (n > 0 ? n : 1)), *iR = malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    int st = OR_OK;
    if (!L || !R || !iL || !iR) { free(L); free(R); free(iL); free(iR); return OR_E_OOM; }
    for (int axis = 0; axis < 3 && st == OR_OK; axis++) {
        if (!(alpha[axis] > 1.0 && alpha[axis] <= 2.0)) { st = OR_E_ARG; break; }
        double gamma = alpha[axis] / 2.0;
        double c = K[axis] / (2.0 * cos(M_PI * alpha[axis] / 2.0));
        for (int64_t q = 0; q < n_g && st == OR_OK; q++) {
            int64_t g = gps[q];
            if (g < 0 || g >= m->n_gp) { st = OR_E_ARG; break; }
            int e1 = or_table_row(m, g, axis, -1, gamma, 0, L);
            int e2 = or_table_row(m, g, axis, +1, gamma, 0, R);
            if (e1 || e2) { st = e1 ? e1 : e2; break; }
            int64_t nl = 0, nr = 0;
            for (int64_t j = 0; j < n; j++) {
                if (L[j] != 0.0) iL[nl++] = j;
                if (R[j] != 0.0) iR[nr++] = j;
            }
            double cw = c * m->gw[g];
            for (int64_t a = 0; a < nl; a++)
                for (int64_t b = 0; b < nr; b++)
                    A[iL[a] * n + iR[b]] += cw * L[iL[a]] * R[iR[b]];
            for (int64_t a = 0; a < nr; a++)
                for (int64_t b = 0; b < nl; b++)
                    A[iR[a] * n + iL[b]] += cw * R[iR[a]] * L[iL[b]];
        }
    }
    free(L); free(R); free(iL); free(iR);
    return st;
}

int or_assemble_form(const or_mesh *m, int axis, double alpha, double beta, int trial_left,
                     const double *c, int all_nodes, double *K)
{
    if (axis < 0 || axis > 2 || !(alpha >= 0.0 && alpha <= 1.0) || !(beta >= 0.0 && beta <= 1.0))
        return OR_E_ARG;
    int64_t n = all_nodes ? m->n_nodes : m->n_dof;
    int64_t nn = n > 0 ? n : 1;
    memset(K, 0, sizeof(double) * n * n);
    double *P = calloc(nn, sizeof(double)), *Q = calloc(nn, sizeof(double));
    int64_t *iP = malloc(sizeof(int64_t) * nn), *iQ = malloc(sizeof(int64_t) * nn);
    if (!P || !Q || !iP || !iQ) { free(P); free(Q); free(iP); free(iQ); return OR_E_OOM; }
    int dtrial = trial_left ? -1 : +1;   /* left operator: the path towards -e_axis */
    for (int64_t g = 0; g < m->n_gp; g++) {
        int e1 = or_table_row(m, g, axis, dtrial, alpha, all_nodes, P);
        int e2 = or_table_row(m, g, axis, -dtrial, beta, all_nodes, Q);
        if (e1 || e2) { free(P); free(Q); free(iP); free(iQ); return e1 ? e1 : e2; }
        int64_t np = 0, nq = 0;
        for (int64_t j = 0; j < n; j++) {
            if (P[j] != 0.0) iP[np++] = j;
            if (Q[j] != 0.0) iQ[nq++] = j;
        }
        double cw = m->gw[g] * (c ? c[g] : 1.0);
        for (int64_t a = 0; a < nq; a++)
            for (int64_t b = 0; b < np; b++)
                K[iQ[a] * n + iP[b]] += cw * Q[iQ[a]] * P[iP[b]];
    }
    free(P); free(Q); free(iP); free(iQ);
    return OR_OK;
}

/* The divergence-form operator with variable coefficients of Section 3 (eq. "equ:sfde2")
 * through its variational form
 *   a(u, v) = - sum_i ( (p_i D_L^{beta_i} u, D_i v) - (q_i D_R^{beta_i} u, D_i v) ),
 * D_i the classical derivative, by the same Gauss quadrature:
 *   A[k][l] = a(psi_l, psi_k)
 *           = - sum_i sum_g w_g D_i psi_k(x_g) (p_i(x_g) D_L psi_l(x_g) - q_i(x_g) D_R psi_l(x_g)).
 * D_i psi_k(x_g) is the order-1 left table row.  beta_i in [0, 1]; p, q: [3][n_gp]
 * coefficient values at the Gauss points.  all_nodes as in or_assemble_form.  A:
 * row-major [n][n]; it is not symmetric. */
int or_assemble_divergence(const or_mesh *m, const double beta[3], const double *p,
                           const double *q, int all_nodes, double *A)
{
    for (int i = 0; i < 3; i++)
        if (!(beta[i] >= 0.0 && beta[i] <= 1.0)) return OR_E_ARG;
    int64_t n = all_nodes ? m->n_nodes : m->n_dof;
    int64_t nn = n > 0 ? n : 1;
    memset(A, 0, sizeof(double) * n * n);
    double *L = calloc(nn, sizeof(double)), *R = calloc(nn, sizeof(double));
    double *D = calloc(nn, sizeof(double));
    if (!L || !R || !D) { free(L); free(R); free(D); return OR_E_OOM; }
    for (int axis = 0; axis < 3; axis++) {
        for (int64_t g = 0; g < m->n_gp; g++) {
            int e1 = or_table_row(m, g, axis, -1, beta[axis], all_nodes, L);
            int e2 = or_table_row(m, g, axis, +1, beta[axis], all_nodes, R);
            int e3 = or_table_row(m, g, axis, -1, 1.0, all_nodes, D);
            if (e1 || e2 || e3) { free(L); free(R); free(D); return e1 ? e1 : (e2 ? e2 : e3); }
            double pw = m->gw[g] * p[axis * m->n_gp + g], qw = m->gw[g] * q[axis * m->n_gp + g];
            for (int64_t k = 0; k < n; k++) {
                if (D[k] == 0.0) continue;
                for (int64_t l = 0; l < n; l++) {
                    double flux = pw * L[l] - qw * R[l];
                    if (flux != 0.0) A[k * n + l] -= D[k] * flux;
                }
            }
        }
    }
    free(L); free(R); free(D);
    return OR_OK;
}

/* Load vector b = M f with the P1 mass matrix M_jk = sum_g w_g phi_j(x_g) phi_k(x_g),
 * j over dofs, k over all nodes.  f: column-major [n_nodes][nrhs]; b: column-major
 * [n_dof][nrhs]. */
int or_load(const or_mesh *m, const double *f, int nrhs, double *b)
{
    memset(b, 0, sizeof(double) * m->n_dof * nrhs);
    double a = rule_a(), bb = rule_b();
    for (int64_t t = 0; t < m->n_tets; t++)
        for (int q = 0; q < 4; q++) {
            double w = m->gw[4 * t + q];
            for (int r = 0; r < nrhs; r++) {
                double fq = 0.0;
                for (int k = 0; k < 4; k++)
                    fq += (k == q ? a : bb) * f[(int64_t)r * m->n_nodes + m->tets[4 * t + k]];
                for (int v = 0; v < 4; v++) {
                    int32_t j = m->dof[m->tets[4 * t + v]];
                    if (j >= 0) b[(int64_t)r * m->n_dof + j] += w * (v == q ? a : bb) * fq;
                }
            }
        }
    return OR_OK;
}

/* Transposed load map: out = M^T lam (nodal), lam column-major [n_dof][nrhs]. */
int or_load_T(const or_mesh *m, const double *lam, int nrhs, double *out)
{
    memset(out, 0, sizeof(double) * m->n_nodes * nrhs);
    double a = rule_a(), bb = rule_b();
    for (int64_t t = 0; t < m->n_tets; t++)
        for (int q = 0; q < 4; q++) {
            double w = m->gw[4 * t + q];
            for (int r = 0; r < nrhs; r++) {
                double lq = 0.0;
                for (int v = 0; v < 4; v++) {
                    int32_t j = m->dof[m->tets[4 * t + v]];
                    if (j >= 0) lq += (v == q ? a : bb) * lam[(int64_t)r * m->n_dof + j];
                }
                for (int k = 0; k < 4; k++)
                    out[(int64_t)r * m->n_nodes + m->tets[4 * t + k]] += w * (k == q ? a : bb) * lq;
            }
        }
    return OR_OK;
}

/* Textbook Cholesky A = L L^T (row-major, lower triangle of Lout filled, upper zero).
 * Returns OR_OK or OR_E_NOT_SPD with *bad_col set. */
int or_cholesky(int64_t n, const double *A, double *Lout, int64_t *bad_col)
{
    memset(Lout, 0, sizeof(double) * n * n);
    for (int64_t j = 0; j < n; j++) {
        double d = A[j * n + j];
        for (int64_t k = 0; k < j; k++) d -= Lout[j * n + k] * Lout[j * n + k];
        if (!(d > 0.0)) { if (bad_col) *bad_col = j; return OR_E_NOT_SPD; }
        double ljj = sqrt(d);
        Lout[j * n + j] = ljj;
        for (int64_t i = j + 1; i < n; i++) {
            double s = A[i * n + j];
            for (int64_t k = 0; k < j; k++) s -= Lout[i * n + k] * Lout[j * n + k];
            Lout[i * n + j] = s / ljj;
        }
    }
    return OR_OK;
}

/* Solve L L^T x = b for nrhs column-major right-hand sides (in place in x). */
void or_chol_solve(int64_t n, const double *L, int nrhs, double *x)
{
    for (int r = 0; r < nrhs; r++) {
        double *y = x + (int64_t)r * n;
        for (int64_t i = 0; i < n; i++) {
            double s = y[i];
            for (int64_t k = 0; k < i; k++) s -= L[i * n + k] * y[k];
            y[i] = s / L[i * n + i];
        }
        for (int64_t i = n - 1; i >= 0; i--) {
            double s = y[i];
            for (int64_t k = i + 1; k < n; k++) s -= L[k * n + i] * y[k];
            y[i] = s / L[i * n + i];
        }
    }
}

/* Per-axis bilinear forms used by the adjoint:
 *   out[i] = s_i sum_g w_g ((L_i lam)_g (R_i u)_g + (R_i lam)_g (L_i u)_g)
 * i.e. lam^T A_i u with A_i the axis-i matrix for K_i = 1. */
int or_axis_forms(const or_mesh *m, const double alpha[3], const double *u, const double *lam,
                  double out[3])
{
    int64_t n = m->n_dof;
    double *L = malloc(sizeof(double) * (n > 0 ? n : 1)), *R = malloc(sizeof(double) * (n > 0 ? n : 1));
    if (!L || !R) { free(L); free(R); return OR_E_OOM; }
    for (int axis = 0; axis < 3; axis++) {
        double gamma = alpha[axis] / 2.0;
        double s = 1.0 / (2.0 * cos(M_PI * alpha[axis] / 2.0));
        double acc = 0.0;
        for (int64_t g = 0; g < m->n_gp; g++) {
            int e1 = or_table_row(m, g, axis, -1, gamma, 0, L);
            int e2 = or_table_row(m, g, axis, +1, gamma, 0, R);
            if (e1 || e2) { free(L); free(R); return e1 ? e1 : e2; }
            double Lu = 0, Ru = 0, Ll = 0, Rl = 0;
            for (int64_t j = 0; j < n; j++) {
                Lu += L[j] * u[j]; Ru += R[j] * u[j];
                Ll += L[j] * lam[j]; Rl += R[j] * lam[j];
            }
            acc += m->gw[g] * (Ll * Ru + Rl * Lu);
        }
        out[axis] = s * acc;
    }
    free(L); free(R);
    return OR_OK;
}
