// Assembly of the subdomain stiffness matrices A^k (FP64) on the GPU.
//
// A^k_ij = sum over ordered element pairs (E, E') inside Omega-hat_k u Gamma^D_k of
//   zeta(E,E')^-1 sum_q w_q |E| int_{E' cap B^h(x_q)} c(x_q, y) (psi_i(y)-psi_i(x_q)) (psi_j(y)-psi_j(x_q)) dy
// (eq. bilinear-multi1 with the quadrature of eq. bil1).  Rule (the same rule as
// the single-domain reference, implemented here from its definition):
//   outer points: 1-D 4-point Gauss-Legendre, 2-D 7-point degree-5 rule on E;
//   inner region: 1-D interval, 2-D l-infinity square clip, or the l2 "nocaps" polygon
//     (vertices of E' in the closed disc plus edge/circle crossings, Fig. approximate-ball e),
//     the "approxcaps" polygon (nocaps plus a chord/arc-midpoint triangle per left-out cap,
//     Fig. approximate-ball f), or, for the whole-element approximate balls (Fig. approximate-ball a-d), all of E'
//     when its barycenter / at least one vertex / at least two vertices lie in the disc;
//   constant kernels: exact polygon moments;
//   fractional / peridynamic kernels: if the bounding boxes of E and E' touch, polar
//     coordinates about x_q with the radial integral in closed form and 8-point
//     Gauss-Legendre in the angle on pieces (split at the edge normal, then each piece
//     ending half-way to +-pi/2); otherwise the 7-point rule on each fan triangle of
//     the polygon.
// On an inner element, psi_i(y) - psi_i(x) = a_i + g_i . (y - x) with g_i the gradient
// of the inner basis and a_i its linear extension at x minus the outer value; the
// inner integral is then a_i a_j S0 + (a_i g_j + a_j g_i) . S1 + g_i^T S2 g_j with
// kernel moments S0, S1, S2 of the region (rank-4 tensors for the vector kernel).
//
// One thread per unordered pair {E, E'} computes both orientations and scatters the
// local matrix, weighted by 1/zeta, into the lower triangle of every A^k holding the
// pair (FP64 atomics) and into the Dirichlet coupling block; a second kernel mirrors
// the lower triangle so every A^k is exactly symmetric.
#include <algorithm>
#include <cmath>

#include "internal.hpp"

namespace nlf {
namespace {

struct AsmArgs {
    const double *xy;
    const int32_t *elems;
    const int8_t *node_dir;
    const uint64_t *mask;     // mask_words words per element: bit k % 64 of word k / 64 = subdomain k
    int mask_words;
    const int32_t *pairs;     // 2 * npairs
    int64_t npairs;
    const int32_t *nodemap;   // K x n_nodes
    int64_t n_nodes;
    const SubdomainDesc *sd;
    double *A;
    double *AD;
    int dim, type, nc;
    double delta, s, c;
    int ball;                 // 0 nocaps, 1 barycenter, 2 123vertices, 3 23vertices, 4 approxcaps (2-D l2)
};

__device__ const double kGLt8[8] = {-0.9602898564975363, -0.7966664774136267, -0.5255324099163290,
                                    -0.1834346424956498, 0.1834346424956498,  0.5255324099163290,
                                    0.7966664774136267,  0.9602898564975363};
__device__ const double kGLw8[8] = {0.1012285362903763, 0.2223810344533745, 0.3137066458778873, 0.3626837833783620,
                                    0.3626837833783620, 0.3137066458778873, 0.2223810344533745, 0.1012285362903763};

struct Rule7 {
    double b[7][3];
    double w[7];
};

__device__ __forceinline__ void rule7(Rule7 &r) {
    const double q15 = sqrt(15.0);
    const double p1 = (6.0 - q15) / 21.0, p2 = (6.0 + q15) / 21.0;
    const double w1 = (155.0 - q15) / 1200.0, w2 = (155.0 + q15) / 1200.0;
    const double c1 = 1.0 - 2.0 * p1, c2 = 1.0 - 2.0 * p2;
    double B[7][3] = {{1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0}, {p1, p1, c1}, {p1, c1, p1}, {c1, p1, p1},
                      {p2, p2, c2}, {p2, c2, p2}, {c2, p2, p2}};
    for (int q = 0; q < 7; ++q) {
        for (int i = 0; i < 3; ++i) r.b[q][i] = B[q][i];
        r.w[q] = q == 0 ? 9.0 / 40.0 : (q < 4 ? w1 : w2);
    }
}

// moments of the kernel over the inner region relative to x
struct Mom {
    double s0;
    double s1[2];
    double s2[3];          // xx, xy, yy
    // vector kernel: T0[ab] (xx,xy,yy), T1[abc] (xxx,xxy,xyy,yyy), T2[abcd] (xxxx,xxxy,xxyy,xyyy,yyyy)
    double t0[3], t1[4], t2[5];
};

__device__ __forceinline__ void mom_zero(Mom &m) {
    m.s0 = 0;
    m.s1[0] = m.s1[1] = 0;
    for (int i = 0; i < 3; ++i) m.s2[i] = 0, m.t0[i] = 0;
    for (int i = 0; i < 4; ++i) m.t1[i] = 0;
    for (int i = 0; i < 5; ++i) m.t2[i] = 0;
}

// add weight * {1, xi, xi xi^T} (scalar kernels)
__device__ __forceinline__ void mom_add_scalar(Mom &m, double w, double ex, double ey) {
    m.s0 += w;
    m.s1[0] += w * ex;
    m.s1[1] += w * ey;
    m.s2[0] += w * ex * ex;
    m.s2[1] += w * ex * ey;
    m.s2[2] += w * ey * ey;
}

// add sum over a direction: f0 th th^T + f1 th th^T th + f2 th th^T th th^T (vector kernel)
__device__ __forceinline__ void mom_add_vec(Mom &m, double f0, double f1, double f2, double cx, double cy) {
    double xx = cx * cx, xy = cx * cy, yy = cy * cy;
    m.t0[0] += f0 * xx; m.t0[1] += f0 * xy; m.t0[2] += f0 * yy;
    m.t1[0] += f1 * xx * cx; m.t1[1] += f1 * xx * cy; m.t1[2] += f1 * xy * cy; m.t1[3] += f1 * yy * cy;
    m.t2[0] += f2 * xx * xx; m.t2[1] += f2 * xx * xy; m.t2[2] += f2 * xx * yy; m.t2[3] += f2 * xy * yy;
    m.t2[4] += f2 * yy * yy;
}

__device__ __forceinline__ double tri_cross(const double *a, const double *b, const double *c) {
    return (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0]);
}

// ---------------------------------------------------------------- region construction
#define MAXV 12

__device__ int clip_axis(double (*P)[2], int n, int ax, double bound, double sgn) {
    double Q[MAXV][2];
    int m = 0;
    for (int k = 0; k < n; ++k) {
        const double *A = P[k], *B = P[(k + 1) % n];
        double fa = sgn * (A[ax] - bound), fb = sgn * (B[ax] - bound);
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

__device__ int region_square(const double (*T)[2], double x0, double x1, double d, double (*P)[2]) {
    for (int k = 0; k < 3; ++k) { P[k][0] = T[k][0]; P[k][1] = T[k][1]; }
    int n = clip_axis(P, 3, 0, x0 + d, 1.0);
    if (n) n = clip_axis(P, n, 0, x0 - d, -1.0);
    if (n) n = clip_axis(P, n, 1, x1 + d, 1.0);
    if (n) n = clip_axis(P, n, 1, x1 - d, -1.0);
    return n >= 3 ? n : 0;
}

// whole-element approximate ball: T itself when selected by the rule, else nothing
__device__ int region_whole(const double (*T)[2], double x0, double x1, double d, int ball, double (*P)[2]) {
    const double rr = d * d;
    int in = 0;
    for (int k = 0; k < 3; ++k) {
        const double dx = T[k][0] - x0, dy = T[k][1] - x1;
        if (dx * dx + dy * dy <= rr) ++in;
    }
    bool take;
    if (ball == 1) {
        const double bx = (T[0][0] + T[1][0] + T[2][0]) / 3.0 - x0, by = (T[0][1] + T[1][1] + T[2][1]) / 3.0 - x1;
        take = bx * bx + by * by <= rr;
    } else {
        take = in >= (ball == 2 ? 1 : 2);
    }
    if (!take) return 0;
    for (int k = 0; k < 3; ++k) {
        P[k][0] = T[k][0];
        P[k][1] = T[k][1];
    }
    return 3;
}

// l2 disc: the vertices of T in the closed disc and the edge/circle crossings strictly
// inside the edges, in boundary order ("nocaps").  With caps, every crossing where the
// boundary leaves the disc (the larger root on its edge) is followed by the point of the
// circle half-way along the arc to the next listed point, x + d (m - x) / |m - x| with m the
// chord midpoint ("approxcaps": each left-out cap becomes the triangle on its chord and arc
// midpoint; a minor arc, inside T, when 2 d exceeds the diameter of T).  At most 9 points:
// an edge adds its start vertex and one crossing, or two crossings, plus one arc point.
__device__ int region_disc(const double (*T)[2], double x0, double x1, double d, bool caps, double (*P)[2]) {
    int n = 0;
    const double rr = d * d;
    bool ex[MAXV];
    for (int k = 0; k < 3; ++k) {
        const double *A = T[k], *B = T[(k + 1) % 3];
        double px = A[0] - x0, py = A[1] - x1, ex_ = B[0] - A[0], ey = B[1] - A[1];
        double aa = px * px + py * py;
        if (aa <= rr) { P[n][0] = A[0]; P[n][1] = A[1]; ex[n] = false; ++n; }
        double qa = ex_ * ex_ + ey * ey, qb = px * ex_ + py * ey, qc = aa - rr;
        double disc = qb * qb - qa * qc;
        if (disc > 0.0) {
            double sq = sqrt(disc);
            double ta = (-qb - sq) / qa, tb = (-qb + sq) / qa;
            if (ta > 0.0 && ta < 1.0) { P[n][0] = A[0] + ta * ex_; P[n][1] = A[1] + ta * ey; ex[n] = false; ++n; }
            if (tb > 0.0 && tb < 1.0) { P[n][0] = A[0] + tb * ex_; P[n][1] = A[1] + tb * ey; ex[n] = true; ++n; }
        }
    }
    if (!caps) return n >= 3 ? n : 0;
    if (n < 2) return 0;
    // insert the arc points from the back, so that each lands after its exit crossing
    int m = n;
    for (int k = 0; k < n; ++k) m += ex[k] ? 1 : 0;
    const double qx = P[0][0], qy = P[0][1];      // the point after the last one
    int w = m;
    for (int k = n - 1; k >= 0; --k) {
        if (ex[k]) {
            const double nx = (k + 1 < n) ? P[k + 1][0] : qx, ny = (k + 1 < n) ? P[k + 1][1] : qy;
            double mx = 0.5 * (P[k][0] + nx) - x0, my = 0.5 * (P[k][1] + ny) - x1;
            double r = sqrt(mx * mx + my * my);
            if (r > 0.0) {
                --w;
                P[w][0] = x0 + d * mx / r;
                P[w][1] = x1 + d * my / r;
            } else {
                --m;            // a chord through x (not possible when 2 d > diam T): no arc point
            }
        }
        --w;
        P[w][0] = P[k][0];
        P[w][1] = P[k][1];
    }
    // w is 0 unless arc points were dropped; close the gap
    if (w > 0)
        for (int k = 0; k < m; ++k) { P[k][0] = P[k + w][0]; P[k][1] = P[k + w][1]; }
    return m >= 3 ? m : 0;
}

// exact moments of a polygon about x (constant kernel), by fan triangles:
// int_T 1 = |T|, int_T xi = |T| centroid, int_T xi xi^T = |T|/12 (sum v v^T + (sum v)(sum v)^T)
__device__ void moments_polygon(const double (*P)[2], int n, double x0, double x1, double c, Mom &m) {
    for (int k = 1; k + 1 < n; ++k) {
        double v[3][2] = {{P[0][0] - x0, P[0][1] - x1}, {P[k][0] - x0, P[k][1] - x1}, {P[k + 1][0] - x0, P[k + 1][1] - x1}};
        double at = 0.5 * ((v[1][0] - v[0][0]) * (v[2][1] - v[0][1]) - (v[1][1] - v[0][1]) * (v[2][0] - v[0][0]));
        double sx = v[0][0] + v[1][0] + v[2][0], sy = v[0][1] + v[1][1] + v[2][1];
        double qxx = v[0][0] * v[0][0] + v[1][0] * v[1][0] + v[2][0] * v[2][0] + sx * sx;
        double qxy = v[0][0] * v[0][1] + v[1][0] * v[1][1] + v[2][0] * v[2][1] + sx * sy;
        double qyy = v[0][1] * v[0][1] + v[1][1] * v[1][1] + v[2][1] * v[2][1] + sy * sy;
        double w = c * at;
        m.s0 += w;
        m.s1[0] += w * sx / 3.0;
        m.s1[1] += w * sy / 3.0;
        m.s2[0] += w * qxx / 12.0;
        m.s2[1] += w * qxy / 12.0;
        m.s2[2] += w * qyy / 12.0;
    }
}

__device__ __forceinline__ double radial(double r, double e) {
    return fabs(e) < 1e-14 ? log(r) : pow(r, e) / e;
}

// separated pair: 7-point rule on each fan triangle with the full kernel
__device__ void moments_fan7(const double (*P)[2], int n, double x0, double x1, const AsmArgs &a, const Rule7 &R,
                             Mom &m) {
    for (int k = 1; k + 1 < n; ++k) {
        const double *p0 = P[0], *p1 = P[k], *p2 = P[k + 1];
        double at = 0.5 * tri_cross(p0, p1, p2);
        for (int q = 0; q < 7; ++q) {
            double yx = R.b[q][0] * p0[0] + R.b[q][1] * p1[0] + R.b[q][2] * p2[0];
            double yy = R.b[q][0] * p0[1] + R.b[q][1] * p1[1] + R.b[q][2] * p2[1];
            double ex = yx - x0, ey = yy - x1;
            double r = sqrt(ex * ex + ey * ey);
            double w = at * R.w[q] * a.c;
            if (a.type == NLFETI_K_FRACTIONAL) {
                mom_add_scalar(m, w * pow(r, -2.0 - 2.0 * a.s), ex, ey);
            } else {
                double cx = ex / r, cy = ey / r;
                double f = w / r;
                mom_add_vec(m, f, f * r, f * r * r, cx, cy);
            }
        }
    }
}

// touching pair: polar rule about x with the geometric angular split
__device__ void moments_polar(const double (*P)[2], int n, double x0, double x1, const AsmArgs &a, Mom &m) {
    const double HALF_PI = 1.5707963267948966;
    for (int k = 0; k < n; ++k) {
        double ux = P[k][0] - x0, uy = P[k][1] - x1;
        double vx = P[(k + 1) % n][0] - x0, vy = P[(k + 1) % n][1] - x1;
        double ex = vx - ux, ey = vy - uy;
        double len = sqrt(ex * ex + ey * ey);
        if (len == 0.0) continue;
        double nx = ey / len, ny = -ex / len;
        double h = nx * ux + ny * uy;
        if (h < 0.0) { nx = -nx; ny = -ny; h = -h; }
        if (h <= 0.0) continue;
        double au = atan2(nx * uy - ny * ux, nx * ux + ny * uy);
        double av = atan2(nx * vy - ny * vx, nx * vx + ny * vy);
        double phi = atan2(ny, nx);
        double sg = av >= au ? 1.0 : -1.0;
        double lo = fmin(au, av), hi = fmax(au, av);
        // pieces: [lo,0],[0,hi] if straddling, each subdivided toward +-pi/2
        double seg[2][2];
        int nseg;
        if (lo < 0.0 && hi > 0.0) { seg[0][0] = lo; seg[0][1] = 0.0; seg[1][0] = 0.0; seg[1][1] = hi; nseg = 2; }
        else { seg[0][0] = lo; seg[0][1] = hi; nseg = 1; }
        int count = 0;
        for (int sgi = 0; sgi < nseg; ++sgi) {
            bool neg = seg[sgi][1] <= 0.0;
            double cur = neg ? -seg[sgi][1] : seg[sgi][0];
            double end = neg ? -seg[sgi][0] : seg[sgi][1];
            while (cur < end && count < 64) {
                double nxt = 0.5 * (cur + HALF_PI);
                if (nxt >= end || count == 63) nxt = end;
                double pa = neg ? -nxt : cur, pb = neg ? -cur : nxt;
                ++count;
                for (int t = 0; t < 8; ++t) {
                    double ps = pa + 0.5 * (pb - pa) * (1.0 + kGLt8[t]);
                    double th = phi + ps;
                    double cth = cos(th), sth = sin(th);
                    double rho = h / cos(ps);
                    double W = a.c * 0.5 * (pb - pa) * kGLw8[t] * sg;
                    if (a.type == NLFETI_K_FRACTIONAL) {
                        double r0 = radial(rho, -2.0 * a.s), r1 = radial(rho, 1.0 - 2.0 * a.s),
                               r2 = radial(rho, 2.0 - 2.0 * a.s);
                        m.s0 += W * r0;
                        m.s1[0] += W * r1 * cth;
                        m.s1[1] += W * r1 * sth;
                        m.s2[0] += W * r2 * cth * cth;
                        m.s2[1] += W * r2 * cth * sth;
                        m.s2[2] += W * r2 * sth * sth;
                    } else {
                        mom_add_vec(m, W * rho, W * 0.5 * rho * rho, W * rho * rho * rho / 3.0, cth, sth);
                    }
                }
                cur = nxt;
            }
        }
    }
}

// local matrix update from moments: acc[i][j] += wt * (a_i a_j S0 + (a_i g_j + a_j g_i).S1 + g_i^T S2 g_j)
template <int NC>
__device__ __forceinline__ void accumulate(double *acc, int ld, int stride, int nl, const double *av,
                                           const double (*g)[2], const Mom &m, double wt) {
    if (NC == 1) {
        for (int i = 0; i < nl; ++i)
            for (int j = 0; j < nl; ++j) {
                double v = av[i] * av[j] * m.s0 + (av[i] * g[j][0] + av[j] * g[i][0]) * m.s1[0] +
                           (av[i] * g[j][1] + av[j] * g[i][1]) * m.s1[1] + g[i][0] * g[j][0] * m.s2[0] +
                           (g[i][0] * g[j][1] + g[i][1] * g[j][0]) * m.s2[1] + g[i][1] * g[j][1] * m.s2[2];
                acc[(i * ld + j) * stride] += wt * v;
            }
    } else {
        // T0[ab], T1[ab c], T2[ab cd] as full small tensors
        double T0[2][2] = {{m.t0[0], m.t0[1]}, {m.t0[1], m.t0[2]}};
        double T1[2][2][2] = {{{m.t1[0], m.t1[1]}, {m.t1[1], m.t1[2]}}, {{m.t1[1], m.t1[2]}, {m.t1[2], m.t1[3]}}};
        double T2[2][2][2][2];
        {
            const double *t = m.t2;
            double v4[2][2][2][2] = {{{{t[0], t[1]}, {t[1], t[2]}}, {{t[1], t[2]}, {t[2], t[3]}}},
                                     {{{t[1], t[2]}, {t[2], t[3]}}, {{t[2], t[3]}, {t[3], t[4]}}}};
            for (int p = 0; p < 16; ++p) (&T2[0][0][0][0])[p] = (&v4[0][0][0][0])[p];
        }
        for (int i = 0; i < nl; ++i)
            for (int j = 0; j < nl; ++j)
                for (int al = 0; al < 2; ++al)
                    for (int be = 0; be < 2; ++be) {
                        double v = av[i] * av[j] * T0[al][be];
                        for (int gm = 0; gm < 2; ++gm) v += (av[i] * g[j][gm] + av[j] * g[i][gm]) * T1[al][be][gm];
                        for (int gm = 0; gm < 2; ++gm)
                            for (int dl = 0; dl < 2; ++dl) v += g[i][gm] * g[j][dl] * T2[al][be][gm][dl];
                        acc[((2 * i + al) * ld + 2 * j + be) * stride] += wt * v;
                    }
    }
}

template <int NC>
__global__ void __launch_bounds__(64) k_assemble(AsmArgs a) {
    extern __shared__ double smem[];
    const int64_t pid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pid >= a.npairs) return;
    const int stride = blockDim.x;
    double *acc = smem + threadIdx.x;
    const int nv = a.dim + 1;
    const int E0 = a.pairs[2 * pid], E1 = a.pairs[2 * pid + 1];
    int nodes[6];
    int nl = 0;
    for (int i = 0; i < nv; ++i) nodes[nl++] = a.elems[(int64_t)E0 * nv + i];
    for (int i = 0; i < nv; ++i) {
        int nd = a.elems[(int64_t)E1 * nv + i];
        bool dup = false;
        for (int j = 0; j < nv; ++j) dup |= (nodes[j] == nd);
        if (!dup) nodes[nl++] = nd;
    }
    const int ld = nl * NC;
    for (int i = 0; i < ld * ld; ++i) acc[i * stride] = 0.0;
    Rule7 R;
    if (a.dim == 2) rule7(R);
    const int ndir = (E0 == E1) ? 1 : 2;
    for (int dir = 0; dir < ndir; ++dir) {
        const int Eo = dir == 0 ? E0 : E1, Ei = dir == 0 ? E1 : E0;
        int io[6], ii[6];
        for (int i = 0; i < nl; ++i) {
            io[i] = -1; ii[i] = -1;
            for (int v = 0; v < nv; ++v) {
                if (a.elems[(int64_t)Eo * nv + v] == nodes[i]) io[i] = v;
                if (a.elems[(int64_t)Ei * nv + v] == nodes[i]) ii[i] = v;
            }
        }
        if (a.dim == 1) {
            double o0 = a.xy[a.elems[2 * (int64_t)Eo]], o1 = a.xy[a.elems[2 * (int64_t)Eo + 1]];
            double i0 = a.xy[a.elems[2 * (int64_t)Ei]], i1 = a.xy[a.elems[2 * (int64_t)Ei + 1]];
            const double q1 = sqrt(3.0 / 7.0 - 2.0 / 7.0 * sqrt(6.0 / 5.0)), q2 = sqrt(3.0 / 7.0 + 2.0 / 7.0 * sqrt(6.0 / 5.0));
            const double w1 = (18.0 + sqrt(30.0)) / 36.0, w2 = (18.0 - sqrt(30.0)) / 36.0;
            const double tq[4] = {-q2, -q1, q1, q2}, wq[4] = {w2, w1, w1, w2};
            double hin = i1 - i0;
            double g[6][2];
            for (int i = 0; i < nl; ++i) {
                g[i][1] = 0.0;
                g[i][0] = ii[i] == 0 ? -1.0 / hin : (ii[i] == 1 ? 1.0 / hin : 0.0);
            }
            for (int q = 0; q < 4; ++q) {
                double lam = 0.5 * (1.0 + tq[q]);
                double x = o0 + (o1 - o0) * lam;
                double lo = fmax(fmin(i0, i1), x - a.delta), hi = fmin(fmax(i0, i1), x + a.delta);
                if (!(hi > lo)) continue;
                double av[6];
                for (int i = 0; i < nl; ++i) {
                    double outv = io[i] == 0 ? 1.0 - lam : (io[i] == 1 ? lam : 0.0);
                    double inv = ii[i] == 0 ? (i1 - x) / hin : (ii[i] == 1 ? (x - i0) / hin : 0.0);
                    av[i] = (Eo == Ei) ? 0.0 : inv - outv;
                }
                Mom m;
                mom_zero(m);
                double dl = lo - x, dh = hi - x;
                m.s0 = a.c * (dh - dl);
                m.s1[0] = a.c * 0.5 * (dh * dh - dl * dl);
                m.s2[0] = a.c * (dh * dh * dh - dl * dl * dl) / 3.0;
                accumulate<NC>(acc, ld, stride, nl, av, g, m, 0.5 * wq[q] * fabs(o1 - o0));
            }
            continue;
        }
        double To[3][2], Ti[3][2];
        for (int v = 0; v < 3; ++v) {
            int no = a.elems[3 * (int64_t)Eo + v], ni = a.elems[3 * (int64_t)Ei + v];
            To[v][0] = a.xy[2 * (int64_t)no]; To[v][1] = a.xy[2 * (int64_t)no + 1];
            Ti[v][0] = a.xy[2 * (int64_t)ni]; Ti[v][1] = a.xy[2 * (int64_t)ni + 1];
        }
        const double areaO = 0.5 * fabs(tri_cross(To[0], To[1], To[2]));
        const double Di = tri_cross(Ti[0], Ti[1], Ti[2]);
        // inner basis: lambda_v(y) = cross(T[v+1]-y, T[v+2]-y) / Di, gradient below
        double g[6][2], l0[6];   // gradient and value at the origin of the inner linear functions
        for (int i = 0; i < nl; ++i) {
            if (ii[i] < 0) { g[i][0] = g[i][1] = 0.0; l0[i] = 0.0; continue; }
            const double *P1 = Ti[(ii[i] + 1) % 3], *P2 = Ti[(ii[i] + 2) % 3];
            g[i][0] = (P1[1] - P2[1]) / Di;
            g[i][1] = (P2[0] - P1[0]) / Di;
            l0[i] = (P1[0] * P2[1] - P1[1] * P2[0]) / Di;
        }
        bool touch;
        {
            double lo0x = fmin(fmin(To[0][0], To[1][0]), To[2][0]), hi0x = fmax(fmax(To[0][0], To[1][0]), To[2][0]);
            double lo0y = fmin(fmin(To[0][1], To[1][1]), To[2][1]), hi0y = fmax(fmax(To[0][1], To[1][1]), To[2][1]);
            double lo1x = fmin(fmin(Ti[0][0], Ti[1][0]), Ti[2][0]), hi1x = fmax(fmax(Ti[0][0], Ti[1][0]), Ti[2][0]);
            double lo1y = fmin(fmin(Ti[0][1], Ti[1][1]), Ti[2][1]), hi1y = fmax(fmax(Ti[0][1], Ti[1][1]), Ti[2][1]);
            double gap = fmax(fmax(lo1x - hi0x, lo0x - hi1x), fmax(lo1y - hi0y, lo0y - hi1y));
            gap = fmax(gap, 0.0);
            touch = gap <= 1e-9 * fmax(hi0x - lo0x, hi0y - lo0y);
        }
        for (int q = 0; q < 7; ++q) {
            double x0 = R.b[q][0] * To[0][0] + R.b[q][1] * To[1][0] + R.b[q][2] * To[2][0];
            double x1 = R.b[q][0] * To[0][1] + R.b[q][1] * To[1][1] + R.b[q][2] * To[2][1];
            double P[MAXV][2];
            int np = (a.type == NLFETI_K_CONST_LINF) ? region_square(Ti, x0, x1, a.delta, P)
                     : (a.ball != 0 && a.ball != 4)   ? region_whole(Ti, x0, x1, a.delta, a.ball, P)
                                                      : region_disc(Ti, x0, x1, a.delta, a.ball == 4, P);
            if (np == 0) continue;
            double av[6];
            for (int i = 0; i < nl; ++i) {
                double outv = io[i] >= 0 ? R.b[q][io[i]] : 0.0;
                double inv = ii[i] >= 0 ? l0[i] + g[i][0] * x0 + g[i][1] * x1 : 0.0;
                av[i] = (Eo == Ei) ? 0.0 : inv - outv;
            }
            Mom m;
            mom_zero(m);
            if (a.type == NLFETI_K_CONST_LINF || a.type == NLFETI_K_CONST_L2) moments_polygon(P, np, x0, x1, a.c, m);
            else if (touch) moments_polar(P, np, x0, x1, a, m);
            else moments_fan7(P, np, x0, x1, a, R, m);
            accumulate<NC>(acc, ld, stride, nl, av, g, m, R.w[q] * areaO);
        }
    }
    // scatter into every subdomain holding the pair
    int zeta = 0;
    for (int w = 0; w < a.mask_words; ++w)
        zeta += __popcll(a.mask[(int64_t)E0 * a.mask_words + w] & a.mask[(int64_t)E1 * a.mask_words + w]);
    const double wz = 1.0 / (double)zeta;
    for (int w = 0; w < a.mask_words; ++w) {
    uint64_t both = a.mask[(int64_t)E0 * a.mask_words + w] & a.mask[(int64_t)E1 * a.mask_words + w];
    while (both) {
        const int k = 64 * w + __ffsll((long long)both) - 1;
        both &= both - 1;
        const SubdomainDesc d = a.sd[k];
        const int32_t *map = a.nodemap + (int64_t)k * a.n_nodes;
        for (int p = 0; p < ld; ++p) {
            int mp = map[nodes[p / NC]];
            if (mp < 0) continue;
            int rp = mp * NC + p % NC;
            for (int q = 0; q < ld; ++q) {
                int mq = map[nodes[q / NC]];
                double v = wz * acc[(p * ld + q) * stride];
                if (mq >= 0) {
                    int cq = mq * NC + q % NC;
                    if (rp >= cq) atomicAdd(a.A + d.offA + (int64_t)rp * d.nk + cq, v);
                } else if (mq <= -2) {
                    int cq = (-2 - mq) * NC + q % NC;
                    atomicAdd(a.AD + d.offAD + (int64_t)rp * d.nD + cq, v);
                }
            }
        }
    }
    }
}

__global__ void k_mirror(double *A, const SubdomainDesc *sd) {
    const SubdomainDesc d = sd[blockIdx.y];
    double *M = A + d.offA;
    const int64_t n = d.nk;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * n; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = t / n, j = t % n;
        if (j > i) M[t] = M[j * n + i];
    }
}

}  // namespace

void assemble_all(nlfeti_problem *p) {
    nlfeti_ctx *c = p->ctx;
    const MeshHost &m = p->mesh;
    // unordered pair list: bounding boxes within delta, sharing a subdomain, not both in the collar
    const int nv = m.dim + 1;
    std::vector<double> lo(m.n_elems * 2, 0.0), hi(m.n_elems * 2, 0.0);
    double ext = 0.0, glo[2] = {INFINITY, INFINITY}, ghi[2] = {-INFINITY, -INFINITY};
    for (int64_t e = 0; e < m.n_elems; ++e) {
        for (int a = 0; a < m.dim; ++a) { lo[2 * e + a] = INFINITY; hi[2 * e + a] = -INFINITY; }
        for (int i = 0; i < nv; ++i) {
            int32_t n = m.elems[e * nv + i];
            for (int a = 0; a < m.dim; ++a) {
                double x = m.xy[(int64_t)n * m.dim + a];
                lo[2 * e + a] = std::min(lo[2 * e + a], x);
                hi[2 * e + a] = std::max(hi[2 * e + a], x);
            }
        }
        for (int a = 0; a < m.dim; ++a) {
            ext = std::max(ext, hi[2 * e + a] - lo[2 * e + a]);
            glo[a] = std::min(glo[a], lo[2 * e + a]);
            ghi[a] = std::max(ghi[a], hi[2 * e + a]);
        }
    }
    const double H = ext > 0 ? ext : 1.0;
    int64_t nb[2] = {1, 1};
    for (int a = 0; a < m.dim; ++a) nb[a] = (int64_t)std::floor((ghi[a] - glo[a]) / H) + 1;
    std::vector<int64_t> start(nb[0] * nb[1] + 1, 0), items(m.n_elems), cell(m.n_elems);
    for (int64_t e = 0; e < m.n_elems; ++e) {
        int64_t cc[2] = {0, 0};
        for (int a = 0; a < m.dim; ++a)
            cc[a] = std::clamp<int64_t>((int64_t)std::floor((lo[2 * e + a] - glo[a]) / H), 0, nb[a] - 1);
        cell[e] = cc[1] * nb[0] + cc[0];
        start[cell[e] + 1]++;
    }
    for (size_t i = 0; i + 1 < start.size(); ++i) start[i + 1] += start[i];
    {
        std::vector<int64_t> fill(start.begin(), start.end() - 1);
        for (int64_t e = 0; e < m.n_elems; ++e) items[fill[cell[e]]++] = e;
    }
    const double r = p->kern.delta;
    std::vector<int32_t> pairs;
    pairs.reserve(1 << 20);
    for (int64_t e = 0; e < m.n_elems; ++e) {
        if (!p->dec.any_sub(e)) continue;
        int64_t clo[2] = {0, 0}, chi[2] = {0, 0};
        for (int a = 0; a < m.dim; ++a) {
            clo[a] = std::max<int64_t>(0, (int64_t)std::floor((lo[2 * e + a] - r - H - glo[a]) / H) - 1);
            chi[a] = std::min<int64_t>(nb[a] - 1, (int64_t)std::floor((hi[2 * e + a] + r - glo[a]) / H) + 1);
        }
        for (int64_t cy = clo[1]; cy <= chi[1]; ++cy)
            for (int64_t cx = clo[0]; cx <= chi[0]; ++cx) {
                int64_t cidx = cy * nb[0] + cx;
                for (int64_t t = start[cidx]; t < start[cidx + 1]; ++t) {
                    int64_t f = items[t];
                    if (f < e) continue;
                    if (!p->dec.share_sub(e, f)) continue;
                    if (m.elem_dir[e] && m.elem_dir[f]) continue;
                    double gap = 0.0;
                    for (int a = 0; a < m.dim; ++a)
                        gap = std::max(gap, std::max(lo[2 * f + a] - hi[2 * e + a], lo[2 * e + a] - hi[2 * f + a]));
                    if (gap > r) continue;
                    pairs.push_back((int32_t)e);
                    pairs.push_back((int32_t)f);
                }
            }
    }
    const int64_t npairs = (int64_t)pairs.size() / 2;
    DevMem d_pairs;
    upload(c, d_pairs, pairs);
    NLF_CUDA(cudaMemsetAsync(p->d_A.p, 0, p->d_A.bytes, c->stream));
    NLF_CUDA(cudaMemsetAsync(p->d_AD.p, 0, p->d_AD.bytes, c->stream));
    AsmArgs a;
    a.xy = p->d_xy.as<double>();
    a.elems = p->d_elems.as<int32_t>();
    a.node_dir = p->d_node_dir.as<int8_t>();
    a.mask = p->d_elem_mask.as<uint64_t>();
    a.mask_words = p->dec.mask_words;
    a.pairs = d_pairs.as<int32_t>();
    a.npairs = npairs;
    a.nodemap = p->d_nodemap.as<int32_t>();
    a.n_nodes = m.n_nodes;
    a.sd = p->d_sd.as<SubdomainDesc>();
    a.A = p->d_A.as<double>();
    a.AD = p->d_AD.as<double>();
    a.dim = m.dim;
    a.type = p->kern.type;
    a.nc = p->nc;
    a.delta = p->kern.delta;
    a.ball = p->kern.ball;
    a.s = p->kern.s;
    a.c = p->kern.scale;
    const int threads = 64;
    if (npairs > 0) {
        const int64_t chunk = 1 << 24;     // keep the grid within limits
        for (int64_t off = 0; off < npairs; off += chunk) {
            AsmArgs b = a;
            b.pairs = a.pairs + 2 * off;
            b.npairs = std::min<int64_t>(chunk, npairs - off);
            unsigned blocks = (unsigned)((b.npairs + threads - 1) / threads);
            if (p->nc == 1) {
                size_t sm = sizeof(double) * 36 * threads;
                k_assemble<1><<<blocks, threads, sm, c->stream>>>(b);
            } else {
                size_t sm = sizeof(double) * 144 * threads;
                NLF_CUDA(cudaFuncSetAttribute(k_assemble<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
                k_assemble<2><<<blocks, threads, sm, c->stream>>>(b);
            }
            NLF_CUDA(cudaGetLastError());
        }
    }
    dim3 grid(64, p->K);
    k_mirror<<<grid, 256, 0, c->stream>>>(p->d_A.as<double>(), p->d_sd.as<SubdomainDesc>());
    NLF_CUDA(cudaGetLastError());
    NLF_CUDA(cudaStreamSynchronize(c->stream));
}

}  // namespace nlf
