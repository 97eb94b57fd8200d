/*
 * FP64 reference quadrature and assembly for the nonlocal stiffness matrix.
 *
 * TEST INFRASTRUCTURE ONLY.  This file belongs to the oracle: plain, slow code
 * written to be checked by eye against the paper.  Only tests, the smoke check
 * and the CPU-baseline leg of the benchmark may load it.  It shares nothing
 * with the CUDA path.
 *
 * What it computes (Sec. 2.3, eq. bil1 and eq. scalarkernel-h; Sec. 3.2,
 * eq. bilinear-multi1; Sec. 6.1, eqs. constantkernel, fractionalkernel,
 * peridynamics):
 *
 *   A_ij = sum over ordered element pairs (E, E') of  w(E,E') *
 *          sum_q  w_q |E|  int_{E' cap B^h(x_q)} c(x_q,y)
 *                 (psi_i(y) - psi_i(x_q)) (psi_j(y) - psi_j(x_q)) dy
 *
 * with x_q the points of a fixed outer rule on E, w(E,E') = 1 for the
 * single-domain matrix and 1/zeta(E,E') for a subdomain matrix (eq. zeta),
 * psi_i(y) the P1 basis evaluated on E' and psi_i(x_q) on E.  The inner
 * region is
 *   1-D: the interval E' cap [x_q - delta, x_q + delta] (exact);
 *   2-D l-infinity: E' clipped by the square of half-width delta (exact);
 *   2-D l2: the "nocaps" polygon of Fig. approximate-ball (e): the vertices
 *           of E' inside the closed disc plus the edge/circle crossings, in
 *           boundary order (the circular caps are left out);
 *   2-D l2, "approxcaps" (ball 4, Fig. approximate-ball f): the nocaps polygon with
 *           each circular cap it leaves out (beyond the chord from a point where the
 *           boundary of E' leaves the disc to the next polygon point) filled by the
 *           triangle on that chord and the midpoint of its arc, a sub-triangle of E'
 *           when 2 delta exceeds the diameter of E' (the arc is then a minor arc);
 *   2-D l2, whole-element approximate balls of Fig. approximate-ball (ball 1-3):
 *           all of E' when its barycenter lies in the closed disc (c), when at
 *           least one of its vertices does (a, b: "123vertices"), or when at
 *           least two of them do (d: "23vertices"); nothing otherwise.
 * Outer rules: 1-D 4-point Gauss-Legendre; 2-D 7-point degree-5 rule.
 * Inner integral:
 *   constant kernels: the integrand is a quadratic polynomial in y, integrated
 *     exactly by a fan triangulation of the polygon and the 3 edge-midpoint rule;
 *   fractional and peridynamic kernels: polar coordinates about x_q, one
 *     triangle (x_q, V_k, V_k+1) per polygon edge (signed), the radial integral
 *     in closed form from r = 0 to the edge, and 8-point Gauss-Legendre in the
 *     polar angle over each edge's angular range.  Lower-limit terms of the
 *     radial antiderivative are dropped: they cancel over a closed polygon that
 *     does not contain x_q, and vanish when it does (then E' = E and the
 *     differences psi(y)-psi(x_q) carry a factor r).
 * Vector kernel (peridynamics): dofs are (node, component), component-minor,
 * kernel c (x-y)(x-y)^T / |x-y|^3.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { K_CONST_LINF = 0, K_CONST_L2 = 1, K_FRACTIONAL = 2, K_PERIDYNAMIC = 3 };

typedef struct {
    int dim;
    int64_t n_nodes;
    const double *xy;          /* dim * n_nodes */
    int64_t n_elems;
    const int32_t *elems;      /* (dim+1) * n_elems */
    const int8_t *node_dir;    /* 1 = Dirichlet node */
    const int8_t *elem_dir;    /* 1 = element in the Dirichlet collar */
} om_mesh;

typedef struct {
    int type;
    double delta;
    double s;
    double c;                  /* kernel constant (already resolved) */
    int ball;                  /* 2-D l2 kernels: 0 nocaps, 1 barycenter, 2 123vertices, 3 23vertices,
                                  4 approxcaps */
} om_kernel;

#define MAXP 16                /* max polygon vertices */
#define MAXL 6                 /* max local nodes of a pair */

/* ---------------------------------------------------------------- outer rules */

static void outer_rule_1d(double a, double b, double xq[4], double wq[4], double bc[4][2]) {
    /* Gauss-Legendre, 4 points on [-1, 1] */
    const double t1 = sqrt(3.0 / 7.0 - 2.0 / 7.0 * sqrt(6.0 / 5.0));
    const double t2 = sqrt(3.0 / 7.0 + 2.0 / 7.0 * sqrt(6.0 / 5.0));
    const double w1 = (18.0 + sqrt(30.0)) / 36.0;
    const double w2 = (18.0 - sqrt(30.0)) / 36.0;
    const double t[4] = {-t2, -t1, t1, t2};
    const double w[4] = {w2, w1, w1, w2};
    for (int q = 0; q < 4; ++q) {
        double lam = 0.5 * (1.0 + t[q]);           /* position in [0,1] */
        xq[q] = a + (b - a) * lam;
        wq[q] = 0.5 * w[q];                         /* weights normalised to sum 1 */
        bc[q][0] = 1.0 - lam;                       /* basis of node 0 (at a) */
        bc[q][1] = lam;                             /* basis of node 1 (at b) */
    }
}

static void outer_rule_2d(const double v[3][2], double xq[7][2], double wq[7], double bc[7][3]) {
    /* 7-point degree-5 rule on a triangle; weights normalised to sum 1 */
    const double r15 = sqrt(15.0);
    const double a1 = (6.0 - r15) / 21.0, a2 = (6.0 + r15) / 21.0;
    const double w0 = 9.0 / 40.0, w1 = (155.0 - r15) / 1200.0, w2 = (155.0 + r15) / 1200.0;
    double B[7][3] = {
        {1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0},
        {a1, a1, 1.0 - 2.0 * a1}, {a1, 1.0 - 2.0 * a1, a1}, {1.0 - 2.0 * a1, a1, a1},
        {a2, a2, 1.0 - 2.0 * a2}, {a2, 1.0 - 2.0 * a2, a2}, {1.0 - 2.0 * a2, a2, a2}};
    double W[7] = {w0, w1, w1, w1, w2, w2, w2};
    for (int q = 0; q < 7; ++q) {
        for (int i = 0; i < 3; ++i) bc[q][i] = B[q][i];
        xq[q][0] = B[q][0] * v[0][0] + B[q][1] * v[1][0] + B[q][2] * v[2][0];
        xq[q][1] = B[q][0] * v[0][1] + B[q][1] * v[1][1] + B[q][2] * v[2][1];
        wq[q] = W[q];
    }
}

/* ------------------------------------------------------- P1 basis on a triangle */

/* lambda_i(y) = (p_{i+1} - y) x (p_{i+2} - y) / D, D = (p1-p0) x (p2-p0) */
static double bary(const double p[3][2], int i, double y0, double y1) {
    const double *a = p[(i + 1) % 3], *b = p[(i + 2) % 3];
    double D = (p[1][0] - p[0][0]) * (p[2][1] - p[0][1]) - (p[1][1] - p[0][1]) * (p[2][0] - p[0][0]);
    double cr = (a[0] - y0) * (b[1] - y1) - (a[1] - y1) * (b[0] - y0);
    return cr / D;
}

static void bary_grad(const double p[3][2], int i, double g[2]) {
    const double *a = p[(i + 1) % 3], *b = p[(i + 2) % 3];
    double D = (p[1][0] - p[0][0]) * (p[2][1] - p[0][1]) - (p[1][1] - p[0][1]) * (p[2][0] - p[0][0]);
    /* d/dy of (a0-y0)(b1-y1) - (a1-y1)(b0-y0) */
    g[0] = (-(b[1]) + a[1]) / D;
    g[1] = (-(a[0]) + b[0]) / D;
}

/* ------------------------------------------------------------------- clipping */

/* keep the part of polygon P with s*(y[ax] - bound) <= 0 */
static int clip_halfplane(double P[MAXP][2], int n, int ax, double bound, double s) {
    double Q[MAXP][2];
    int m = 0;
    for (int k = 0; k < n; ++k) {
        const double *A = P[k], *B = P[(k + 1) % n];
        double fa = s * (A[ax] - bound), fb = s * (B[ax] - bound);
        if (fa <= 0.0) { Q[m][0] = A[0]; Q[m][1] = A[1]; ++m; }
        if ((fa < 0.0 && fb > 0.0) || (fa > 0.0 && fb < 0.0)) {
            double t = fa / (fa - fb);
            Q[m][0] = A[0] + t * (B[0] - A[0]);
            Q[m][1] = A[1] + t * (B[1] - A[1]);
            ++m;
        }
    }
    for (int k = 0; k < m; ++k) { P[k][0] = Q[k][0]; P[k][1] = Q[k][1]; }
    return m;
}

static int clip_square(const double tri[3][2], const double x[2], double d, double P[MAXP][2]) {
    int n = 3;
    for (int k = 0; k < 3; ++k) { P[k][0] = tri[k][0]; P[k][1] = tri[k][1]; }
    n = clip_halfplane(P, n, 0, x[0] + d, 1.0);
    if (n) n = clip_halfplane(P, n, 0, x[0] - d, -1.0);
    if (n) n = clip_halfplane(P, n, 1, x[1] + d, 1.0);
    if (n) n = clip_halfplane(P, n, 1, x[1] - d, -1.0);
    return n < 3 ? 0 : n;
}

/* Walk the boundary of the triangle in order and list the vertices inside the closed disc
 * and the edge/circle crossings strictly inside the edges.  exit_[k] = 1 marks a crossing
 * where the boundary leaves the disc (the larger root on its edge). */
static int disc_walk(const double tri[3][2], const double x[2], double d, double P[MAXP][2], int exit_[MAXP]) {
    int n = 0;
    double d2 = d * d;
    for (int k = 0; k < 3; ++k) {
        const double *A = tri[k], *B = tri[(k + 1) % 3];
        double ax = A[0] - x[0], ay = A[1] - x[1];
        double ex = B[0] - A[0], ey = B[1] - A[1];
        if (ax * ax + ay * ay <= d2) { P[n][0] = A[0]; P[n][1] = A[1]; exit_[n] = 0; ++n; }
        double qa = ex * ex + ey * ey;
        double qb = ax * ex + ay * ey;
        double qc = ax * ax + ay * ay - d2;
        double disc = qb * qb - qa * qc;
        if (disc > 0.0) {
            double sq = sqrt(disc);
            double t1 = (-qb - sq) / qa, t2 = (-qb + sq) / qa;
            if (t1 > 0.0 && t1 < 1.0) { P[n][0] = A[0] + t1 * ex; P[n][1] = A[1] + t1 * ey; exit_[n] = 0; ++n; }
            if (t2 > 0.0 && t2 < 1.0) { P[n][0] = A[0] + t2 * ex; P[n][1] = A[1] + t2 * ey; exit_[n] = 1; ++n; }
        }
    }
    return n;
}

/* nocaps polygon: vertices inside the closed disc plus edge/circle crossings, in order */
static int clip_disc_nocaps(const double tri[3][2], const double x[2], double d, double P[MAXP][2]) {
    int exit_[MAXP];
    int n = disc_walk(tri, x, d, P, exit_);
    return n < 3 ? 0 : n;
}

/* approxcaps polygon: the nocaps walk, and after every exit crossing the point of the circle
 * half-way along the arc to the next listed point (x + d (m - x) / |m - x|, m the chord
 * midpoint), so that each left-out cap is replaced by the triangle on its chord and arc
 * midpoint.  A circle entering and leaving E' through one edge yields that triangle alone. */
static int clip_disc_approxcaps(const double tri[3][2], const double x[2], double d, double P[MAXP][2]) {
    double W[MAXP][2];
    int exit_[MAXP];
    int n = disc_walk(tri, x, d, W, exit_);
    if (n < 2) return 0;
    int m = 0;
    for (int k = 0; k < n; ++k) {
        P[m][0] = W[k][0]; P[m][1] = W[k][1]; ++m;
        if (!exit_[k]) continue;
        const double *Q = W[(k + 1) % n];
        double mx = 0.5 * (W[k][0] + Q[0]) - x[0], my = 0.5 * (W[k][1] + Q[1]) - x[1];
        double r = sqrt(mx * mx + my * my);
        if (r > 0.0) { P[m][0] = x[0] + d * mx / r; P[m][1] = x[1] + d * my / r; ++m; }
    }
    return m < 3 ? 0 : m;
}

/* ------------------------------------------------------- local pair structure */

typedef struct {
    int nl;                    /* local nodes */
    int32_t node[MAXL];
    double a_out[MAXL];        /* psi_i(x_q) evaluated on the outer element E */
    int in_inner[MAXL];        /* index 0..2 in E' or -1 */
} pairloc;

static void pair_nodes(const om_mesh *M, int64_t e, int64_t ep, pairloc *L) {
    int nv = M->dim + 1;
    L->nl = 0;
    for (int i = 0; i < nv; ++i) { L->node[L->nl] = M->elems[e * nv + i]; L->in_inner[L->nl] = -1; L->nl++; }
    for (int i = 0; i < nv; ++i) {
        int32_t nd = M->elems[ep * nv + i];
        int found = -1;
        for (int j = 0; j < L->nl; ++j) if (L->node[j] == nd) found = j;
        if (found < 0) { L->node[L->nl] = nd; L->in_inner[L->nl] = i; L->nl++; }
        else L->in_inner[found] = i;
    }
}

/* ------------------------------------------------------------ 1-D pair matrix */

static void pair_1d(const om_mesh *M, const om_kernel *K, int64_t e, int64_t ep, pairloc *L, double *out) {
    int nl = L->nl;
    double a = M->xy[M->elems[2 * e]], b = M->xy[M->elems[2 * e + 1]];
    double c0 = M->xy[M->elems[2 * ep]], c1 = M->xy[M->elems[2 * ep + 1]];
    double xq[4], wq[4], bc[4][2];
    outer_rule_1d(a, b, xq, wq, bc);
    double len = fabs(b - a);
    for (int q = 0; q < 4; ++q) {
        for (int i = 0; i < nl; ++i) L->a_out[i] = (i < 2) ? bc[q][i] : 0.0;
        double lo = fmax(fmin(c0, c1), xq[q] - K->delta);
        double hi = fmin(fmax(c0, c1), xq[q] + K->delta);
        if (!(hi > lo)) continue;
        /* Simpson's rule is exact for the quadratic integrand */
        double ys[3] = {lo, 0.5 * (lo + hi), hi};
        double ws[3] = {(hi - lo) / 6.0, 4.0 * (hi - lo) / 6.0, (hi - lo) / 6.0};
        for (int t = 0; t < 3; ++t) {
            double dv[MAXL];
            for (int i = 0; i < nl; ++i) {
                double inner = 0.0;
                if (L->in_inner[i] == 0) inner = (c1 - ys[t]) / (c1 - c0);
                if (L->in_inner[i] == 1) inner = (ys[t] - c0) / (c1 - c0);
                dv[i] = inner - L->a_out[i];
            }
            double wt = wq[q] * len * ws[t] * K->c;
            for (int i = 0; i < nl; ++i)
                for (int j = 0; j < nl; ++j) out[i * nl + j] += wt * dv[i] * dv[j];
        }
    }
}

/* ------------------------------------------------------------ 2-D pair matrix */

static double rad_antider(double r, double e) {
    /* antiderivative of r^(e-1): r^e / e, or log r when e == 0 */
    if (fabs(e) < 1e-14) return log(r);
    return pow(r, e) / e;
}

/* Angular pieces of [lo, hi] (angles from the edge normal, inside (-pi/2, pi/2)): split at 0,
 * then each piece ends half-way between its start and +-pi/2 (clipped to the interval). */
static int angle_pieces(double lo, double hi, double *plo, double *phi, int cap) {
    const double H = 1.5707963267948966;
    int n = 0;
    double segs[2][2];
    int ns = 0;
    if (lo < 0.0 && hi > 0.0) { segs[0][0] = lo; segs[0][1] = 0.0; segs[1][0] = 0.0; segs[1][1] = hi; ns = 2; }
    else { segs[0][0] = lo; segs[0][1] = hi; ns = 1; }
    for (int s = 0; s < ns; ++s) {
        double a = segs[s][0], b = segs[s][1];
        int neg = (b <= 0.0);
        double x = neg ? -b : a, e = neg ? -a : b;       /* work on the non-negative side */
        while (x < e && n < cap) {
            double nxt = 0.5 * (x + H);
            if (nxt >= e || n == cap - 1) nxt = e;
            if (neg) { plo[n] = -nxt; phi[n] = -x; }
            else { plo[n] = x; phi[n] = nxt; }
            ++n;
            x = nxt;
        }
    }
    return n;
}

/* elements whose bounding boxes touch or overlap (l-infinity gap below 1e-9 of the outer extent) */
static int elems_touch(const om_mesh *M, int64_t e, int64_t ep) {
    double lo0[2], hi0[2], lo1[2], hi1[2];
    for (int a = 0; a < 2; ++a) { lo0[a] = lo1[a] = 1e300; hi0[a] = hi1[a] = -1e300; }
    for (int i = 0; i < 3; ++i) {
        int32_t n0 = M->elems[3 * e + i], n1 = M->elems[3 * ep + i];
        for (int a = 0; a < 2; ++a) {
            double x0 = M->xy[2 * n0 + a], x1 = M->xy[2 * n1 + a];
            if (x0 < lo0[a]) lo0[a] = x0;
            if (x0 > hi0[a]) hi0[a] = x0;
            if (x1 < lo1[a]) lo1[a] = x1;
            if (x1 > hi1[a]) hi1[a] = x1;
        }
    }
    double ext = fmax(hi0[0] - lo0[0], hi0[1] - lo0[1]);
    double gap = 0.0;
    for (int a = 0; a < 2; ++a) gap = fmax(gap, fmax(lo1[a] - hi0[a], lo0[a] - hi1[a]));
    return gap <= 1e-9 * ext;
}

/* inner integral at one outer point x: for every local (i, j),
 *   out[i, j] += weight * int_{E' cap B^h(x)} c(x,y) (psi_i(y) - a_i)(psi_j(y) - a_j) dy
 * with psi_i the P1 basis of the inner triangle w (zero for nodes not in it) and
 * a_i the outer values psi_i(x).  same_elem marks E' = E (then psi_i(y) - a_i vanishes at y = x). */
static void inner_2d(const om_kernel *K, const double w[3][2], const double x[2], const pairloc *L, int same_elem,
                     int near, double weight, double *out) {
    int nl = L->nl, nc = (K->type == K_PERIDYNAMIC) ? 2 : 1;
    int ldo = nl * nc;
    double g[MAXL][2];
    for (int i = 0; i < nl; ++i) {
        if (L->in_inner[i] >= 0) bary_grad(w, L->in_inner[i], g[i]);
        else { g[i][0] = 0.0; g[i][1] = 0.0; }
    }
    double P[MAXP][2];
    int np;
    if (K->type == K_CONST_LINF) np = clip_square(w, x, K->delta, P);
    else if (K->ball == 0) np = clip_disc_nocaps(w, x, K->delta, P);
    else if (K->ball == 4) np = clip_disc_approxcaps(w, x, K->delta, P);
    else {
        /* whole-element ball: E' itself or nothing */
        int inside = 0;
        double bx = 0.0, by = 0.0;
        for (int v = 0; v < 3; ++v) {
            double dx = w[v][0] - x[0], dy = w[v][1] - x[1];
            if (dx * dx + dy * dy <= K->delta * K->delta) ++inside;
            bx += w[v][0] / 3.0;
            by += w[v][1] / 3.0;
        }
        int take;
        if (K->ball == 1) take = (bx - x[0]) * (bx - x[0]) + (by - x[1]) * (by - x[1]) <= K->delta * K->delta;
        else if (K->ball == 2) take = inside >= 1;
        else take = inside >= 2;
        np = 0;
        if (take)
            for (int v = 0; v < 3; ++v) { P[v][0] = w[v][0]; P[v][1] = w[v][1]; np = 3; }
    }
    if (np < 3) return;
    if (K->type == K_CONST_LINF || K->type == K_CONST_L2) {
        /* fan triangulation + edge-midpoint rule (exact for quadratics) */
        for (int k = 1; k + 1 < np; ++k) {
            const double *p0 = P[0], *p1 = P[k], *p2 = P[k + 1];
            double At = 0.5 * ((p1[0] - p0[0]) * (p2[1] - p0[1]) - (p1[1] - p0[1]) * (p2[0] - p0[0]));
            double mids[3][2] = {{0.5 * (p0[0] + p1[0]), 0.5 * (p0[1] + p1[1])},
                                 {0.5 * (p1[0] + p2[0]), 0.5 * (p1[1] + p2[1])},
                                 {0.5 * (p2[0] + p0[0]), 0.5 * (p2[1] + p0[1])}};
            for (int t = 0; t < 3; ++t) {
                double dv[MAXL];
                for (int i = 0; i < nl; ++i) {
                    double inner = (L->in_inner[i] >= 0) ? bary(w, L->in_inner[i], mids[t][0], mids[t][1]) : 0.0;
                    dv[i] = inner - L->a_out[i];
                }
                double wt = weight * At / 3.0 * K->c;
                for (int i = 0; i < nl; ++i)
                    for (int j = 0; j < nl; ++j) out[i * ldo + j] += wt * dv[i] * dv[j];
            }
        }
        return;
    }
    double ai[MAXL];
    for (int i = 0; i < nl; ++i) {
        double inner = (L->in_inner[i] >= 0) ? bary(w, L->in_inner[i], x[0], x[1]) : 0.0;
        ai[i] = same_elem ? 0.0 : inner - L->a_out[i];   /* psi(y)-psi(x) = r g.theta on E itself */
    }
    if (!near) {
        /* separated pair: 7-point rule on each fan triangle of the polygon, full singular integrand */
        for (int k = 1; k + 1 < np; ++k) {
            double T[3][2] = {{P[0][0], P[0][1]}, {P[k][0], P[k][1]}, {P[k + 1][0], P[k + 1][1]}};
            double At = 0.5 * ((T[1][0] - T[0][0]) * (T[2][1] - T[0][1]) - (T[1][1] - T[0][1]) * (T[2][0] - T[0][0]));
            double yq[7][2], wy[7], by[7][3];
            outer_rule_2d(T, yq, wy, by);
            for (int t = 0; t < 7; ++t) {
                double ex = yq[t][0] - x[0], ey = yq[t][1] - x[1];
                double r = sqrt(ex * ex + ey * ey);
                double dv[MAXL];
                for (int i = 0; i < nl; ++i) {
                    double inner = (L->in_inner[i] >= 0) ? bary(w, L->in_inner[i], yq[t][0], yq[t][1]) : 0.0;
                    dv[i] = inner - L->a_out[i];
                }
                double W = weight * At * wy[t] * K->c;
                if (K->type == K_FRACTIONAL) {
                    double kr = pow(r, -2.0 - 2.0 * K->s);
                    for (int i = 0; i < nl; ++i)
                        for (int j = 0; j < nl; ++j) out[i * ldo + j] += W * kr * dv[i] * dv[j];
                } else {
                    double th2[2] = {ex / r, ey / r};
                    for (int i = 0; i < nl; ++i)
                        for (int j = 0; j < nl; ++j)
                            for (int al = 0; al < 2; ++al)
                                for (int be = 0; be < 2; ++be)
                                    out[(2 * i + al) * ldo + 2 * j + be] += W / r * th2[al] * th2[be] * dv[i] * dv[j];
                }
            }
        }
        return;
    }
    /* touching pair: polar coordinates about x, one signed triangle per polygon edge; the
     * angular range of each edge, measured from the edge normal, is split at the normal and
     * then geometrically toward +-pi/2 (each piece ends half-way to +-pi/2), with 8-point
     * Gauss-Legendre on every piece */
    static const double gt[8] = {-0.9602898564975363, -0.7966664774136267, -0.5255324099163290,
                                 -0.1834346424956498, 0.1834346424956498, 0.5255324099163290,
                                 0.7966664774136267, 0.9602898564975363};
    static const double gw[8] = {0.1012285362903763, 0.2223810344533745, 0.3137066458778873,
                                 0.3626837833783620, 0.3626837833783620, 0.3137066458778873,
                                 0.2223810344533745, 0.1012285362903763};
    for (int k = 0; k < np; ++k) {
        double ux = P[k][0] - x[0], uy = P[k][1] - x[1];
        double vx = P[(k + 1) % np][0] - x[0], vy = P[(k + 1) % np][1] - x[1];
        double ex = vx - ux, ey = vy - uy;
        double el = sqrt(ex * ex + ey * ey);
        if (el == 0.0) continue;
        double nx = ey / el, ny = -ex / el;          /* unit normal of the edge line */
        double dist = nx * ux + ny * uy;
        if (dist < 0.0) { nx = -nx; ny = -ny; dist = -dist; }
        if (dist <= 0.0) continue;                   /* x on the edge line: zero-measure triangle */
        double psu = atan2(nx * uy - ny * ux, nx * ux + ny * uy);   /* angle of u from the normal */
        double psv = atan2(nx * vy - ny * vx, nx * vx + ny * vy);
        double phi = atan2(ny, nx);
        double sgn = psv >= psu ? 1.0 : -1.0;
        double lo = psv >= psu ? psu : psv, hi = psv >= psu ? psv : psu;
        double plo[64], phi_[64];
        int npc = angle_pieces(lo, hi, plo, phi_, 64);
        for (int pc = 0; pc < npc; ++pc) {
            double a = plo[pc], b = phi_[pc];
            for (int t = 0; t < 8; ++t) {
                double ps = a + 0.5 * (b - a) * (1.0 + gt[t]);
                double th = phi + ps;
                double ct = cos(th), st = sin(th);
                double rho = dist / cos(ps);
                double W = weight * K->c * 0.5 * (b - a) * gw[t] * sgn;
                double gth[MAXL];
                for (int i = 0; i < nl; ++i) gth[i] = g[i][0] * ct + g[i][1] * st;
                if (K->type == K_FRACTIONAL) {
                    double s = K->s;
                    double R0 = rad_antider(rho, -2.0 * s);
                    double R1 = rad_antider(rho, 1.0 - 2.0 * s);
                    double R2 = rad_antider(rho, 2.0 - 2.0 * s);
                    for (int i = 0; i < nl; ++i)
                        for (int j = 0; j < nl; ++j)
                            out[i * ldo + j] += W * (ai[i] * ai[j] * R0 + (ai[i] * gth[j] + ai[j] * gth[i]) * R1 +
                                                     gth[i] * gth[j] * R2);
                } else {
                    double R0 = rho, R1 = 0.5 * rho * rho, R2 = rho * rho * rho / 3.0;
                    double th2[2] = {ct, st};
                    for (int i = 0; i < nl; ++i)
                        for (int j = 0; j < nl; ++j) {
                            double val = W * (ai[i] * ai[j] * R0 + (ai[i] * gth[j] + ai[j] * gth[i]) * R1 +
                                              gth[i] * gth[j] * R2);
                            for (int al = 0; al < 2; ++al)
                                for (int be = 0; be < 2; ++be)
                                    out[(2 * i + al) * ldo + 2 * j + be] += val * th2[al] * th2[be];
                        }
                }
            }
        }
    }
}

static void elem_tri(const om_mesh *M, int64_t e, double v[3][2]) {
    for (int i = 0; i < 3; ++i) {
        int32_t n0 = M->elems[3 * e + i];
        v[i][0] = M->xy[2 * n0]; v[i][1] = M->xy[2 * n0 + 1];
    }
}

static void pair_2d(const om_mesh *M, const om_kernel *K, int64_t e, int64_t ep, pairloc *L, double *out) {
    int nl = L->nl;
    double v[3][2], w[3][2];
    elem_tri(M, e, v);
    elem_tri(M, ep, w);
    double areaE = 0.5 * fabs((v[1][0] - v[0][0]) * (v[2][1] - v[0][1]) - (v[1][1] - v[0][1]) * (v[2][0] - v[0][0]));
    double xq[7][2], wq[7], bc[7][3];
    outer_rule_2d(v, xq, wq, bc);
    int near = elems_touch(M, e, ep);
    for (int q = 0; q < 7; ++q) {
        for (int i = 0; i < nl; ++i) L->a_out[i] = (i < 3) ? bc[q][i] : 0.0;
        inner_2d(K, w, xq[q], L, e == ep, near, wq[q] * areaE, out);
    }
}

/* Inner integral of the ordered pair (E = e, E' = ep) at an arbitrary point x (2-D only), with
 * psi_i(x) taken as the linear extension of E's basis.  Exposed for brute-force checks. */
int oracle_point_integral(const om_mesh *M, const om_kernel *K, int64_t e, int64_t ep, double x0, double x1,
                          double *out, int32_t *nodes_out) {
    pairloc L;
    pair_nodes(M, e, ep, &L);
    int nc = (K->type == K_PERIDYNAMIC) ? 2 : 1;
    int ldo = L.nl * nc;
    memset(out, 0, sizeof(double) * ldo * ldo);
    double v[3][2], w[3][2], x[2] = {x0, x1};
    elem_tri(M, e, v);
    elem_tri(M, ep, w);
    for (int i = 0; i < L.nl; ++i) L.a_out[i] = (i < 3) ? bary(v, i, x0, x1) : 0.0;
    inner_2d(K, w, x, &L, e == ep, elems_touch(M, e, ep), 1.0, out);
    for (int i = 0; i < L.nl; ++i) nodes_out[i] = L.node[i];
    return L.nl;
}

/* Local matrix of the ordered pair (E = e outer, E' = ep inner).  Local dofs are
 * (node, component) component-minor over the node list written to nodes_out.
 * Returns the number of local nodes; out receives (nl*nc)^2 values (row-major). */
int oracle_pair_matrix(const om_mesh *M, const om_kernel *K, int64_t e, int64_t ep, double *out, int32_t *nodes_out) {
    pairloc L;
    pair_nodes(M, e, ep, &L);
    int nc = (K->type == K_PERIDYNAMIC) ? 2 : 1;
    int ldo = L.nl * nc;
    memset(out, 0, sizeof(double) * ldo * ldo);
    if (M->dim == 1) pair_1d(M, K, e, ep, &L, out);
    else pair_2d(M, K, e, ep, &L, out);
    for (int i = 0; i < L.nl; ++i) nodes_out[i] = L.node[i];
    return L.nl;
}

/* ------------------------------------------------------------ neighbour search */

typedef struct {
    double lo[2], hi[2];
} bbox;

static void elem_bbox(const om_mesh *M, int64_t e, bbox *b) {
    int nv = M->dim + 1;
    for (int a = 0; a < M->dim; ++a) { b->lo[a] = 1e300; b->hi[a] = -1e300; }
    for (int i = 0; i < nv; ++i) {
        int32_t nd = M->elems[e * nv + i];
        for (int a = 0; a < M->dim; ++a) {
            double x = M->xy[nd * M->dim + a];
            if (x < b->lo[a]) b->lo[a] = x;
            if (x > b->hi[a]) b->hi[a] = x;
        }
    }
}

/* plain bucket grid over bbox lower corners, bucket width H >= max element extent */
typedef struct {
    int dim;
    double org[2], H;
    int64_t nb[2];
    int64_t *start;            /* nb0*nb1 + 1 */
    int64_t *items;
    bbox *bb;
} bucket_grid;

static void grid_build(const om_mesh *M, bucket_grid *G) {
    G->dim = M->dim;
    G->bb = (bbox *)malloc(sizeof(bbox) * M->n_elems);
    double lo[2] = {1e300, 1e300}, hi[2] = {-1e300, -1e300}, ext = 0.0;
    for (int64_t e = 0; e < M->n_elems; ++e) {
        elem_bbox(M, e, &G->bb[e]);
        for (int a = 0; a < M->dim; ++a) {
            if (G->bb[e].lo[a] < lo[a]) lo[a] = G->bb[e].lo[a];
            if (G->bb[e].hi[a] > hi[a]) hi[a] = G->bb[e].hi[a];
            double x = G->bb[e].hi[a] - G->bb[e].lo[a];
            if (x > ext) ext = x;
        }
    }
    G->H = ext > 0 ? ext : 1.0;
    for (int a = 0; a < 2; ++a) {
        G->org[a] = (a < M->dim) ? lo[a] : 0.0;
        G->nb[a] = (a < M->dim) ? (int64_t)floor((hi[a] - lo[a]) / G->H) + 1 : 1;
    }
    int64_t nbt = G->nb[0] * G->nb[1];
    G->start = (int64_t *)calloc(nbt + 1, sizeof(int64_t));
    G->items = (int64_t *)malloc(sizeof(int64_t) * M->n_elems);
    int64_t *cell = (int64_t *)malloc(sizeof(int64_t) * M->n_elems);
    for (int64_t e = 0; e < M->n_elems; ++e) {
        int64_t c[2] = {0, 0};
        for (int a = 0; a < M->dim; ++a) {
            c[a] = (int64_t)floor((G->bb[e].lo[a] - G->org[a]) / G->H);
            if (c[a] < 0) c[a] = 0;
            if (c[a] >= G->nb[a]) c[a] = G->nb[a] - 1;
        }
        cell[e] = c[1] * G->nb[0] + c[0];
        G->start[cell[e] + 1]++;
    }
    for (int64_t i = 0; i < nbt; ++i) G->start[i + 1] += G->start[i];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * nbt);
    for (int64_t i = 0; i < nbt; ++i) fill[i] = G->start[i];
    for (int64_t e = 0; e < M->n_elems; ++e) G->items[fill[cell[e]]++] = e;
    free(fill);
    free(cell);
}

static void grid_free(bucket_grid *G) {
    free(G->start); free(G->items); free(G->bb);
}

/* all elements whose bbox is within l-infinity distance r of bbox b (ascending element id) */
static int64_t grid_query(const bucket_grid *G, const bbox *b, double r, int64_t *out, int64_t cap) {
    int64_t lo[2] = {0, 0}, hi[2] = {0, 0};
    for (int a = 0; a < G->dim; ++a) {
        lo[a] = (int64_t)floor((b->lo[a] - r - G->H - G->org[a]) / G->H) - 1;
        hi[a] = (int64_t)floor((b->hi[a] + r - G->org[a]) / G->H) + 1;
        if (lo[a] < 0) lo[a] = 0;
        if (hi[a] >= G->nb[a]) hi[a] = G->nb[a] - 1;
    }
    int64_t n = 0;
    for (int64_t cy = lo[1]; cy <= hi[1]; ++cy)
        for (int64_t cx = lo[0]; cx <= hi[0]; ++cx) {
            int64_t c = cy * G->nb[0] + cx;
            for (int64_t t = G->start[c]; t < G->start[c + 1]; ++t) {
                int64_t e = G->items[t];
                const bbox *o = &G->bb[e];
                int ok = 1;
                for (int a = 0; a < G->dim; ++a) {
                    double gap = fmax(0.0, fmax(o->lo[a] - b->hi[a], b->lo[a] - o->hi[a]));
                    if (gap > r) ok = 0;
                }
                if (ok) { if (n < cap) out[n] = e; ++n; }
            }
        }
    /* insertion sort for a deterministic order */
    int64_t m = n < cap ? n : cap;
    for (int64_t i = 1; i < m; ++i) {
        int64_t x = out[i], j = i - 1;
        while (j >= 0 && out[j] > x) { out[j + 1] = out[j]; --j; }
        out[j + 1] = x;
    }
    return n;
}

static int popcount64(uint64_t x) {
    int c = 0;
    while (x) { x &= x - 1; ++c; }
    return c;
}

/* element e in subdomain k: bit k % 64 of word k / 64 of its mask (W words per element) */
static int mask_has(const uint64_t *elem_mask, int W, int64_t e, int k) {
    return (int)((elem_mask[e * W + k / 64] >> (k % 64)) & 1u);
}

/* zeta(E, E'): the number of subdomains holding both elements */
static int mask_common(const uint64_t *elem_mask, int W, int64_t e, int64_t ep) {
    int c = 0;
    for (int w = 0; w < W; ++w) c += popcount64(elem_mask[e * W + w] & elem_mask[ep * W + w]);
    return c;
}

/* ------------------------------------------------------------------- assembly */

/*
 * Assemble sum over ordered element pairs into A.
 *   elem_mask : per element W words, bit k % 64 of word k / 64 set when the element belongs
 *               to subdomain k (Omega-hat_k union Gamma^D_k); may be NULL when k < 0.
 *   k         : subdomain index (pairs with both bits set, weight 1/zeta(E,E'))
 *               or -1 (all pairs, weight 1).
 *   dof_of    : (n_nodes*nc) local dof index of (node, comp), or -1.
 *   mode 0    : A is dense n_dofs x n_dofs row-major.
 *   mode 1    : A is the lower band (kd+1) x n_dofs, A[(i-j)*n_dofs + j] = A_ij, i>=j.
 *   g, Bg     : optional; for columns that are Dirichlet nodes, Bg[row] += A_row,col * g[col]
 *               (g indexed by node*nc + comp).  A may be NULL to compute Bg only.
 * Pairs of two Dirichlet elements are skipped: all their nodes are Dirichlet.
 * Returns 0 on success, -1 on a band overflow.
 */
int oracle_assemble(const om_mesh *M, const om_kernel *K, const uint64_t *elem_mask, int W, int k,
                    const int32_t *dof_of, int64_t n_dofs, int mode, int64_t kd, double *A,
                    const double *g, double *Bg, int nthreads) {
    int nc = (K->type == K_PERIDYNAMIC) ? 2 : 1;
    bucket_grid G;
    grid_build(M, &G);
    const int64_t cap = 1 << 16;
    int status = 0;
    int64_t chunk = 64;
    int maxld = MAXL * nc;
    /* per outer element: compute all local matrices (parallel), then scatter in order (serial) */
    int64_t nE = M->n_elems;
    int64_t **nbr = (int64_t **)calloc(chunk, sizeof(int64_t *));
    int64_t *nnb = (int64_t *)calloc(chunk, sizeof(int64_t));
    double **loc = (double **)calloc(chunk, sizeof(double *));
    int32_t **locn = (int32_t **)calloc(chunk, sizeof(int32_t *));
    int **locnl = (int **)calloc(chunk, sizeof(int *));
    for (int64_t c0 = 0; c0 < nE; c0 += chunk) {
        int64_t c1 = c0 + chunk < nE ? c0 + chunk : nE;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
        for (int64_t e = c0; e < c1; ++e) {
            int64_t slot = e - c0;
            int64_t *list = (int64_t *)malloc(sizeof(int64_t) * cap);
            int64_t n = 0;
            int use = 1;
            if (k >= 0 && !mask_has(elem_mask, W, e, k)) use = 0;
            if (use) n = grid_query(&G, &G.bb[e], K->delta, list, cap);
            if (n > cap) n = cap;
            nnb[slot] = 0;
            nbr[slot] = list;
            loc[slot] = (double *)malloc(sizeof(double) * (n > 0 ? n : 1) * maxld * maxld);
            locn[slot] = (int32_t *)malloc(sizeof(int32_t) * (n > 0 ? n : 1) * MAXL);
            locnl[slot] = (int *)malloc(sizeof(int) * (n > 0 ? n : 1));
            int64_t kept = 0;
            for (int64_t t = 0; t < n; ++t) {
                int64_t ep = list[t];
                if (M->elem_dir[e] && M->elem_dir[ep]) continue;
                if (k >= 0 && !mask_has(elem_mask, W, ep, k)) continue;
                list[kept] = ep;
                locnl[slot][kept] = oracle_pair_matrix(M, K, e, ep, loc[slot] + kept * maxld * maxld,
                                                       locn[slot] + kept * MAXL);
                ++kept;
            }
            nnb[slot] = kept;
        }
        for (int64_t e = c0; e < c1; ++e) {
            int64_t slot = e - c0;
            for (int64_t t = 0; t < nnb[slot]; ++t) {
                int64_t ep = nbr[slot][t];
                double wgt = 1.0;
                if (k >= 0) wgt = 1.0 / (double)mask_common(elem_mask, W, e, ep);
                int nl = locnl[slot][t];
                int ld = nl * nc;
                const double *L = loc[slot] + t * maxld * maxld;
                const int32_t *nodes = locn[slot] + t * MAXL;
                for (int a = 0; a < ld; ++a) {
                    int32_t ra = dof_of[nodes[a / nc] * nc + a % nc];
                    if (ra < 0) continue;
                    for (int b = 0; b < ld; ++b) {
                        int32_t nb_node = nodes[b / nc];
                        int32_t cb = dof_of[nb_node * nc + b % nc];
                        double val = wgt * L[a * ld + b];
                        if (cb >= 0) {
                            if (!A) continue;                  /* only the Dirichlet term was asked for */
                            if (mode == 0) A[(int64_t)ra * n_dofs + cb] += val;
                            else if (ra >= cb) {
                                if (ra - cb > kd) status = -1;
                                else A[(int64_t)(ra - cb) * n_dofs + cb] += val;
                            }
                        } else if (g && Bg && M->node_dir[nb_node]) {
                            Bg[ra] += val * g[nb_node * nc + b % nc];
                        }
                    }
                }
            }
            free(nbr[slot]); free(loc[slot]); free(locn[slot]); free(locnl[slot]);
        }
    }
    free(nbr); free(nnb); free(loc); free(locn); free(locnl);
    grid_free(&G);
    return status;
}

/*
 * Rows of the single-domain matrix for selected dofs, without assembling the rest:
 * out[r * ncols + col] for every dof column (n_nodes*nc columns, Dirichlet included).
 * A_ij collects the pairs (E, E') whose union of nodes contains node(i).
 */
int oracle_assemble_rows(const om_mesh *M, const om_kernel *K, const int64_t *rows, int64_t nrows, double *out,
                         int nthreads) {
    int nc = (K->type == K_PERIDYNAMIC) ? 2 : 1;
    int64_t ncols = M->n_nodes * nc;
    bucket_grid G;
    grid_build(M, &G);
    int nv = M->dim + 1;
    const int64_t cap = 1 << 16;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int64_t r = 0; r < nrows; ++r) {
        int64_t dof = rows[r];
        int32_t node = (int32_t)(dof / nc);
        int comp = (int)(dof % nc);
        double *row = out + r * ncols;
        int64_t *list = (int64_t *)malloc(sizeof(int64_t) * cap);
        double L[MAXL * 2 * MAXL * 2];   /* room for the vector kernel */
        int32_t nodes[MAXL];
        for (int64_t t = 0; t < M->n_elems; ++t) {
            int has = 0;
            for (int i = 0; i < nv; ++i) if (M->elems[t * nv + i] == node) has = 1;
            if (!has) continue;
            int64_t n = grid_query(&G, &G.bb[t], K->delta, list, cap);
            if (n > cap) n = cap;
            for (int64_t s = 0; s < n; ++s) {
                int64_t o = list[s];
                /* pair (t, o): t contains node */
                for (int pass = 0; pass < 2; ++pass) {
                    int64_t e = pass == 0 ? t : o, ep = pass == 0 ? o : t;
                    if (pass == 1) {
                        /* (o, t) with o containing node was already counted from o's side */
                        int oh = 0;
                        for (int i = 0; i < nv; ++i) if (M->elems[o * nv + i] == node) oh = 1;
                        if (oh) continue;
                    }
                    if (M->elem_dir[e] && M->elem_dir[ep]) continue;
                    int nl = oracle_pair_matrix(M, K, e, ep, L, nodes);
                    int ld = nl * nc;
                    int a = -1;
                    for (int i = 0; i < nl; ++i) if (nodes[i] == node) a = i * nc + comp;
                    if (a < 0) continue;
                    for (int b = 0; b < ld; ++b) row[(int64_t)nodes[b / nc] * nc + b % nc] += L[a * ld + b];
                }
            }
        }
        free(list);
    }
    grid_free(&G);
    return 0;
}
