/* oracle.c — plain, slow FP64 CPU oracle of the meshless porous-media solvers of
 * Strzelczyk, Rot, Kosec & Matyka, "Cross-validation of meshless Navier-Stokes
 * solvers in porous media flows" (arXiv 2404.14195).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg load this file's library.  It shares no code, header, table or
 * helper with the CUDA library; the two meet only at the seeded node clouds.
 *
 * Everything is FP64, compiled with -ffp-contract=off (no fused multiply-add), in
 * the order the paper states each step.  Node loops are parallelised with OpenMP
 * where each node's result is independent of the others; reductions are serial.
 *
 * Parity pins for each routine live in the tests: polynomial reproduction and sum
 * rules (weights), the pure-polynomial limit N_L = N_p (textbook 7-point stencils),
 * exact reproduction of a PHS basis function, finite differences of the
 * interpolation weights (derivative right-hand sides), high-precision null-space
 * solves on tiny stencils, brute-force neighbour lists, collision invariants,
 * the lattice-shift limit of the streaming step and the analytic Poiseuille flow.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXN 128   /* max saddle-system size N_L + N_p */
#define ORC_MAXOPS 32  /* max right-hand sides per stencil */

/* ---- geometry --------------------------------------------------------------
 * Periodic cell of side d = 1: the displacement between two points is taken to
 * the nearest periodic image ("periodic search of stencils' members", case
 * definition section). */
static double orc_mimg(double d) { return d - rint(d); }

/* ---- stencils: the N_L nearest nodes (meshless discretisation section) -------
 * For every query point, S(1..N_L) are the N_L nodes closest by periodic
 * distance, ordered by (squared distance, node index).  When the query is a node
 * its own index comes first (distance zero), so S_i(1) = i as the augmented
 * system assumes.  Brute force over all nodes.                                  */
int orc_knn(int64_t n, const double *xyz, int64_t nq, const double *q, int n_l, int32_t *out) {
    if (n_l < 1 || n_l > n) return -1;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t a = 0; a < nq; ++a) {
        double bd[ORC_MAXN];
        int64_t bi[ORC_MAXN];
        int cnt = 0;
        for (int64_t j = 0; j < n; ++j) {
            double dx = orc_mimg(xyz[3 * j] - q[3 * a]);
            double dy = orc_mimg(xyz[3 * j + 1] - q[3 * a + 1]);
            double dz = orc_mimg(xyz[3 * j + 2] - q[3 * a + 2]);
            double d2 = dx * dx + dy * dy + dz * dz;
            if (cnt == n_l && (d2 > bd[cnt - 1] || (d2 == bd[cnt - 1] && j > bi[cnt - 1]))) continue;
            int pos = (cnt < n_l) ? cnt++ : cnt - 1;
            while (pos > 0 && (bd[pos - 1] > d2 || (bd[pos - 1] == d2 && bi[pos - 1] > j))) {
                bd[pos] = bd[pos - 1];
                bi[pos] = bi[pos - 1];
                --pos;
            }
            bd[pos] = d2;
            bi[pos] = j;
        }
        if (cnt < n_l) bad = 1;
        for (int t = 0; t < n_l; ++t) out[a * n_l + t] = (int32_t)bi[t];
    }
    return bad ? -2 : 0;
}

/* Same neighbour lists as orc_knn, found through a uniform periodic cell grid:
 * every node within distance R of the query is examined (all cells overlapping
 * the ball), and R is doubled until the n_l-th best distance is below R, so no
 * unexamined node can be closer or tie.  Used for large clouds. */
int orc_knn_grid(int64_t n, const double *xyz, int64_t nq, const double *q, int n_l, int32_t *out) {
    if (n_l < 1 || n_l > n || n_l > ORC_MAXN) return -1;
    int G = (int)cbrt((double)n / 8.0);
    if (G < 1) G = 1;
    if (G > 256) G = 256;
    const double cs = 1.0 / G;
    int64_t ncell = (int64_t)G * G * G;
    int64_t *head = malloc(sizeof(int64_t) * ncell), *next = malloc(sizeof(int64_t) * n);
    for (int64_t c = 0; c < ncell; ++c) head[c] = -1;
    for (int64_t j = n - 1; j >= 0; --j) {
        int a = (int)(xyz[3 * j] * G), b = (int)(xyz[3 * j + 1] * G), c = (int)(xyz[3 * j + 2] * G);
        a = a < 0 ? 0 : (a >= G ? G - 1 : a); b = b < 0 ? 0 : (b >= G ? G - 1 : b); c = c < 0 ? 0 : (c >= G ? G - 1 : c);
        int64_t cell = ((int64_t)a * G + b) * G + c;
        next[j] = head[cell];
        head[cell] = j;
    }
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t t = 0; t < nq; ++t) {
        double bd[ORC_MAXN];
        int64_t bi[ORC_MAXN];
        double qx = q[3 * t] - floor(q[3 * t]), qy = q[3 * t + 1] - floor(q[3 * t + 1]), qz = q[3 * t + 2] - floor(q[3 * t + 2]);
        int ca = (int)(qx * G), cb = (int)(qy * G), cc = (int)(qz * G);
        ca = ca >= G ? G - 1 : ca; cb = cb >= G ? G - 1 : cb; cc = cc >= G ? G - 1 : cc;
        for (double R = 1.5 * cs;; R *= 2.0) {
            int reach = (int)ceil(R / cs);
            int full = 2 * reach + 1 >= G;
            int lo = full ? 0 : -reach, hi = full ? G - 1 : reach;
            int cnt = 0;
            for (int da = lo; da <= hi; ++da)
                for (int db = lo; db <= hi; ++db)
                    for (int dc = lo; dc <= hi; ++dc) {
                        int a = full ? da : ((ca + da) % G + G) % G;
                        int b = full ? db : ((cb + db) % G + G) % G;
                        int c = full ? dc : ((cc + dc) % G + G) % G;
                        for (int64_t j = head[((int64_t)a * G + b) * G + c]; j >= 0; j = next[j]) {
                            double dx = orc_mimg(xyz[3 * j] - qx), dy = orc_mimg(xyz[3 * j + 1] - qy);
                            double dz = orc_mimg(xyz[3 * j + 2] - qz);
                            double d2 = dx * dx + dy * dy + dz * dz;
                            if (cnt == n_l && (d2 > bd[cnt - 1] || (d2 == bd[cnt - 1] && j > bi[cnt - 1]))) continue;
                            int pos = (cnt < n_l) ? cnt++ : cnt - 1;
                            while (pos > 0 && (bd[pos - 1] > d2 || (bd[pos - 1] == d2 && bi[pos - 1] > j))) {
                                bd[pos] = bd[pos - 1]; bi[pos] = bi[pos - 1]; --pos;
                            }
                            bd[pos] = d2; bi[pos] = j;
                        }
                    }
            if ((cnt == n_l && bd[n_l - 1] < R * R) || full) {
                if (cnt < n_l) bad = 1;
                for (int k = 0; k < n_l; ++k) out[t * n_l + k] = (int32_t)(k < cnt ? bi[k] : 0);
                break;
            }
        }
    }
    free(head); free(next);
    return bad ? -2 : 0;
}

/* ---- RBF-FD weights (Eqs. operatorApprox, rbfScaling, augmentedSystem) -------
 * Basis: polyharmonic spline Phi(r) = r^k (odd k) in the scaled distance
 * r / delta_i, augmented with the N_p = C(m+3, 3) monomials of total degree <= m
 * in the scaled displacement (x - x_c) / delta_i, listed in graded lexicographic
 * order {1, x, y, z, x^2, xy, xz, y^2, yz, z^2, ...} as in the paper's footnote.
 * The saddle system [[A, P], [P^T, 0]] [w; lambda] = [b; c] is solved per stencil
 * and operator; lambda is discarded.                                            */

/* exponent triples of the monomials of degree <= m, graded lexicographic */
int orc_monomials(int m, int *ex) {
    int np = 0;
    for (int d = 0; d <= m; ++d)
        for (int a = d; a >= 0; --a)
            for (int b = d - a; b >= 0; --b) {
                ex[3 * np] = a;
                ex[3 * np + 1] = b;
                ex[3 * np + 2] = d - a - b;
                ++np;
            }
    return np;
}

static double orc_ipow(double x, int e) {
    double r = 1.0;
    for (int i = 0; i < e; ++i) r *= x;
    return r;
}

/* Operator kinds: the linear operator L applied to the basis and evaluated at the
 * point y = x_c + offset. */
enum { ORC_OP_INTERP = 0, ORC_OP_DX = 1, ORC_OP_DY = 2, ORC_OP_DZ = 3, ORC_OP_LAP = 4 };

/* L applied to the RBF centred at stencil node j, evaluated at the scaled point eta:
 * s = eta - xi_j (scaled), rho = |s|.  Derivatives are with respect to physical
 * coordinates, hence the 1/delta and 1/delta^2 factors.                         */
static double orc_rbf_rhs(int kind, int k, const double s[3], double delta) {
    double rho = sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
    switch (kind) {
    case ORC_OP_INTERP: return orc_ipow(rho, k);
    case ORC_OP_DX: case ORC_OP_DY: case ORC_OP_DZ:
        /* d/dy_a (|y - x_j| / delta)^k = k rho^(k-2) s_a / delta */
        return (double)k * orc_ipow(rho, k - 2) * s[kind - ORC_OP_DX] / delta;
    case ORC_OP_LAP:
        /* Laplacian of rho^k in three dimensions: k (k + 1) rho^(k-2), over delta^2 */
        return (double)k * (double)(k + 1) * orc_ipow(rho, k - 2) / (delta * delta);
    }
    return NAN;
}

/* L applied to the monomial x^a y^b z^c (scaled coordinates) at eta. */
static double orc_mono_rhs(int kind, const int e[3], const double eta[3], double delta) {
    switch (kind) {
    case ORC_OP_INTERP:
        return orc_ipow(eta[0], e[0]) * orc_ipow(eta[1], e[1]) * orc_ipow(eta[2], e[2]);
    case ORC_OP_DX: case ORC_OP_DY: case ORC_OP_DZ: {
        int ax = kind - ORC_OP_DX;
        if (e[ax] == 0) return 0.0;
        double v = (double)e[ax] / delta;
        for (int t = 0; t < 3; ++t) v *= orc_ipow(eta[t], t == ax ? e[t] - 1 : e[t]);
        return v;
    }
    case ORC_OP_LAP: {
        double sum = 0.0;
        for (int ax = 0; ax < 3; ++ax) {
            if (e[ax] < 2) continue;
            double v = (double)e[ax] * (double)(e[ax] - 1);
            for (int t = 0; t < 3; ++t) v *= orc_ipow(eta[t], t == ax ? e[t] - 2 : e[t]);
            sum += v;
        }
        return sum / (delta * delta);
    }
    }
    return NAN;
}

/* LU factorisation with partial pivoting, in place (row-major n x n).  Returns 0,
 * or 1 when a pivot is exactly zero. */
static int orc_lu(int n, double *a, int *piv) {
    for (int c = 0; c < n; ++c) {
        int p = c;
        double best = fabs(a[c * n + c]);
        for (int r = c + 1; r < n; ++r)
            if (fabs(a[r * n + c]) > best) { best = fabs(a[r * n + c]); p = r; }
        piv[c] = p;
        if (best == 0.0) return 1;
        if (p != c)
            for (int t = 0; t < n; ++t) { double tmp = a[c * n + t]; a[c * n + t] = a[p * n + t]; a[p * n + t] = tmp; }
        for (int r = c + 1; r < n; ++r) {
            double l = a[r * n + c] / a[c * n + c];
            a[r * n + c] = l;
            for (int t = c + 1; t < n; ++t) a[r * n + t] -= l * a[c * n + t];
        }
    }
    return 0;
}

static void orc_lu_solve(int n, const double *lu, const int *piv, double *x) {
    for (int c = 0; c < n; ++c)
        if (piv[c] != c) { double t = x[c]; x[c] = x[piv[c]]; x[piv[c]] = t; }
    for (int r = 1; r < n; ++r)
        for (int t = 0; t < r; ++t) x[r] -= lu[r * n + t] * x[t];
    for (int r = n - 1; r >= 0; --r) {
        for (int t = r + 1; t < n; ++t) x[r] -= lu[r * n + t] * x[t];
        x[r] /= lu[r * n + r];
    }
}

/* Weights for nc stencils.
 *   xyz (n x 3) node positions; centre (nc x 3) stencil centres x_c;
 *   centre_is_node: 1 when x_c is the node S(1) itself, so that delta (the local
 *     scaling of Eq. rbfScaling) is the distance to the nearest other node S(2);
 *     0 for free points (probes), delta = distance to S(1);
 *   idx (nc x n_l) stencils; k PHS order; m monomial order;
 *   op_kind / op_off (n_ops, n_ops x 3): operator L and the offset y - x_c;
 *   w (nc x n_ops x n_l) output; refine: iterative-refinement steps with the
 *   residual accumulated in long double.
 * Returns the number of singular systems. */
int orc_rbf_weights(int64_t n, const double *xyz, int64_t nc, const double *centre,
                    int centre_is_node, int n_l, const int32_t *idx, int k, int m, int n_ops,
                    const int *op_kind, const double *op_off, int refine, double *w) {
    (void)n;
    int ex[3 * 64];
    int np = orc_monomials(m, ex);
    int ns = n_l + np;
    if (ns > ORC_MAXN || n_ops > ORC_MAXOPS || n_l < np) return -1;
    int n_sing = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : n_sing)
    for (int64_t i = 0; i < nc; ++i) {
        double *M = (double *)malloc(sizeof(double) * ns * ns * 2);
        double *LU = M + ns * ns;
        double xi[ORC_MAXN][3];
        int piv[ORC_MAXN];
        const double *xc = centre + 3 * i;
        for (int j = 0; j < n_l; ++j) {
            int64_t g = idx[i * n_l + j];
            for (int a = 0; a < 3; ++a) xi[j][a] = orc_mimg(xyz[3 * g + a] - xc[a]);
        }
        int jd = centre_is_node ? 1 : 0;
        double delta = sqrt(xi[jd][0] * xi[jd][0] + xi[jd][1] * xi[jd][1] + xi[jd][2] * xi[jd][2]);
        for (int j = 0; j < n_l; ++j)
            for (int a = 0; a < 3; ++a) xi[j][a] /= delta;
        /* assemble [[A, P], [P^T, 0]] */
        for (int r = 0; r < ns; ++r)
            for (int c = 0; c < ns; ++c) {
                double v;
                if (r < n_l && c < n_l) {
                    double s[3] = {xi[r][0] - xi[c][0], xi[r][1] - xi[c][1], xi[r][2] - xi[c][2]};
                    v = orc_rbf_rhs(ORC_OP_INTERP, k, s, delta);
                } else if (r < n_l) {
                    v = orc_mono_rhs(ORC_OP_INTERP, ex + 3 * (c - n_l), xi[r], delta);
                } else if (c < n_l) {
                    v = orc_mono_rhs(ORC_OP_INTERP, ex + 3 * (r - n_l), xi[c], delta);
                } else {
                    v = 0.0;
                }
                M[r * ns + c] = v;
            }
        memcpy(LU, M, sizeof(double) * ns * ns);
        int sing = orc_lu(ns, LU, piv);
        n_sing += sing;
        for (int o = 0; o < n_ops; ++o) {
            double eta[3] = {op_off[3 * o] / delta, op_off[3 * o + 1] / delta, op_off[3 * o + 2] / delta};
            double rhs[ORC_MAXN], x[ORC_MAXN], d[ORC_MAXN];
            for (int j = 0; j < n_l; ++j) {
                double s[3] = {eta[0] - xi[j][0], eta[1] - xi[j][1], eta[2] - xi[j][2]};
                rhs[j] = orc_rbf_rhs(op_kind[o], k, s, delta);
            }
            for (int l = 0; l < np; ++l) rhs[n_l + l] = orc_mono_rhs(op_kind[o], ex + 3 * l, eta, delta);
            double *wo = w + (i * n_ops + o) * n_l;
            if (sing) {
                for (int j = 0; j < n_l; ++j) wo[j] = NAN;
                continue;
            }
            memcpy(x, rhs, sizeof(double) * ns);
            orc_lu_solve(ns, LU, piv, x);
            for (int it = 0; it < refine; ++it) {
                for (int r = 0; r < ns; ++r) {
                    long double acc = rhs[r];
                    for (int c = 0; c < ns; ++c) acc -= (long double)M[r * ns + c] * (long double)x[c];
                    d[r] = (double)acc;
                }
                orc_lu_solve(ns, LU, piv, d);
                for (int r = 0; r < ns; ++r) x[r] += d[r];
            }
            for (int j = 0; j < n_l; ++j) wo[j] = x[j];
        }
        free(M);
    }
    return n_sing;
}

/* ---- meshless Navier-Stokes, artificial compressibility (MNS section) ------
 * One step, per Eqs. MNS_intermediate, MNS_pressure, MNS_velocity, MNS_C and the
 * MNS algorithm of the appendix:
 *   v' = v + dt (nu lap v - (v . grad) v + g)            at fluid nodes, v' = 0 on walls
 *   repeat n_p times:
 *     p <- p - dt C^2 rho div v                          at fluid nodes
 *     wall p from dp/dn = 0 (Neumann BC): p_b solves n . grad p = 0 discretised on
 *       the wall node's Neumann stencil {b, N_L - 1 nearest fluid nodes}, so it
 *       reads only the just-updated fluid p
 *     v <- v' - dt/rho grad p                            at fluid nodes, v = 0 on walls
 *     C = beta max(max_i |v_i|, v_ref)
 * The first divergence uses v'.  C at entry is beta max(max_i |v_i|, v_ref) of the
 * velocity passed in.  w4 holds per node (n x 4 x n_l) the weights of d/dx, d/dy,
 * d/dz and the Laplacian.  The nb wall nodes wl[] have Neumann stencils idxb
 * (nb x n_l, the wall node first) with gradient weights wgb (nb x 3 x n_l).
 * prm = {nu, gx, gy, gz, dt, beta, v_ref, rho}.
 * res (nsteps) receives |v_new - v_old|_2 / |v_new|_2 over fluid nodes per step. */
int orc_acm_run(int64_t n, const uint8_t *type, const double *nrm, int n_l, const int32_t *idx,
                const double *w4, int64_t nb, const int32_t *wl, const int32_t *idxb,
                const double *wgb, const double *prm, int n_p, int nsteps, double *u, double *v,
                double *w, double *p, double *res) {
    const double nu = prm[0], gx = prm[1], gy = prm[2], gz = prm[3], dt = prm[4], beta = prm[5],
                 vref = prm[6], rho = prm[7];
    double *us = malloc(sizeof(double) * n), *vs = malloc(sizeof(double) * n), *ws = malloc(sizeof(double) * n);
    double *uo = malloc(sizeof(double) * n), *vo = malloc(sizeof(double) * n), *wo = malloc(sizeof(double) * n);
    double *pn = malloc(sizeof(double) * n);
    double vmax = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double s = sqrt(u[i] * u[i] + v[i] * v[i] + w[i] * w[i]);
        if (s > vmax) vmax = s;
    }
    double C = beta * (vmax > vref ? vmax : vref);
    for (int step = 0; step < nsteps; ++step) {
        memcpy(uo, u, sizeof(double) * n); memcpy(vo, v, sizeof(double) * n); memcpy(wo, w, sizeof(double) * n);
        /* intermediate velocity, Eq. MNS_intermediate */
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            if (type[i]) { us[i] = vs[i] = ws[i] = 0.0; continue; }
            const double *wx = w4 + (i * 4 + 0) * n_l, *wy = w4 + (i * 4 + 1) * n_l;
            const double *wz = w4 + (i * 4 + 2) * n_l, *wl = w4 + (i * 4 + 3) * n_l;
            double g[3][4] = {{0}}; /* [component][dx, dy, dz, lap] */
            for (int j = 0; j < n_l; ++j) {
                int64_t s = idx[i * n_l + j];
                double f[3] = {u[s], v[s], w[s]};
                for (int c = 0; c < 3; ++c) {
                    g[c][0] += wx[j] * f[c];
                    g[c][1] += wy[j] * f[c];
                    g[c][2] += wz[j] * f[c];
                    g[c][3] += wl[j] * f[c];
                }
            }
            double vel[3] = {u[i], v[i], w[i]}, gg[3] = {gx, gy, gz}, out[3];
            for (int c = 0; c < 3; ++c) {
                double adv = vel[0] * g[c][0] + vel[1] * g[c][1] + vel[2] * g[c][2];
                out[c] = vel[c] + dt * (nu * g[c][3] - adv + gg[c]);
            }
            us[i] = out[0]; vs[i] = out[1]; ws[i] = out[2];
        }
        memcpy(u, us, sizeof(double) * n); memcpy(v, vs, sizeof(double) * n); memcpy(w, ws, sizeof(double) * n);
        for (int it = 0; it < n_p; ++it) {
            /* pressure, Eq. MNS_pressure, at fluid nodes */
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < n; ++i) {
                if (type[i]) { pn[i] = p[i]; continue; }
                const double *wx = w4 + (i * 4 + 0) * n_l, *wy = w4 + (i * 4 + 1) * n_l, *wz = w4 + (i * 4 + 2) * n_l;
                double div = 0.0;
                for (int j = 0; j < n_l; ++j) {
                    int64_t s = idx[i * n_l + j];
                    div += wx[j] * u[s] + wy[j] * v[s] + wz[j] * w[s];
                }
                pn[i] = p[i] - dt * C * C * rho * div;
            }
            /* wall pressure from the Neumann condition n . grad p = 0 */
#pragma omp parallel for schedule(static)
            for (int64_t b = 0; b < nb; ++b) {
                int64_t i = wl[b];
                const double *wx = wgb + (b * 3 + 0) * n_l, *wy = wgb + (b * 3 + 1) * n_l, *wz = wgb + (b * 3 + 2) * n_l;
                const double *nn = nrm + 3 * i;
                double self = nn[0] * wx[0] + nn[1] * wy[0] + nn[2] * wz[0];
                double acc = 0.0;
                for (int j = 1; j < n_l; ++j) {
                    double wn = nn[0] * wx[j] + nn[1] * wy[j] + nn[2] * wz[j];
                    acc += wn * pn[idxb[b * n_l + j]];
                }
                pn[i] = -acc / self;
            }
            memcpy(p, pn, sizeof(double) * n);
            /* velocity correction, Eq. MNS_velocity, and the speed of sound, Eq. MNS_C */
            vmax = 0.0;
#pragma omp parallel for schedule(static) reduction(max : vmax)
            for (int64_t i = 0; i < n; ++i) {
                if (type[i]) { u[i] = v[i] = w[i] = 0.0; continue; }
                const double *wx = w4 + (i * 4 + 0) * n_l, *wy = w4 + (i * 4 + 1) * n_l, *wz = w4 + (i * 4 + 2) * n_l;
                double gp[3] = {0.0, 0.0, 0.0};
                for (int j = 0; j < n_l; ++j) {
                    double ps = p[idx[i * n_l + j]];
                    gp[0] += wx[j] * ps;
                    gp[1] += wy[j] * ps;
                    gp[2] += wz[j] * ps;
                }
                u[i] = us[i] - dt / rho * gp[0];
                v[i] = vs[i] - dt / rho * gp[1];
                w[i] = ws[i] - dt / rho * gp[2];
                double s = sqrt(u[i] * u[i] + v[i] * v[i] + w[i] * w[i]);
                if (s > vmax) vmax = s;
            }
            C = beta * (vmax > vref ? vmax : vref);
        }
        if (res) {
            double dn = 0.0, nn = 0.0;
            for (int64_t i = 0; i < n; ++i) {
                if (type[i]) continue;
                double a = u[i] - uo[i], b = v[i] - vo[i], c = w[i] - wo[i];
                dn += a * a + b * b + c * c;
                nn += u[i] * u[i] + v[i] * v[i] + w[i] * w[i];
            }
            res[step] = nn > 0.0 ? sqrt(dn) / sqrt(nn) : 0.0;
        }
    }
    free(us); free(vs); free(ws); free(uo); free(vo); free(wo); free(pn);
    return 0;
}

/* ---- meshless lattice Boltzmann, TRT (MLBM section) -------------------------
 * Velocity set e (q x 3, integers as doubles), weights omega (q), opposite index
 * opp (q).  Lattice speed of sound c_s^2 = 1/3. */

/* Macroscopic variables, Eq. macro_var: rho = sum f, v = sum f e / rho. */
static void orc_lbm_moments(int q, const double *e, const double *f, int64_t n, int64_t i,
                            double *rho, double vel[3]) {
    double r = 0.0, m[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < q; ++k) {
        double fk = f[(int64_t)k * n + i];
        r += fk;
        m[0] += fk * e[3 * k]; m[1] += fk * e[3 * k + 1]; m[2] += fk * e[3 * k + 2];
    }
    *rho = r;
    vel[0] = m[0] / r; vel[1] = m[1] / r; vel[2] = m[2] / r;
}

/* Second-order equilibrium, Eq. feq, c_s^2 = 1/3. */
static double orc_feq(const double *e, const double *omega, int k, double rho, const double v[3]) {
    const double cs2 = 1.0 / 3.0;
    double ev = e[3 * k] * v[0] + e[3 * k + 1] * v[1] + e[3 * k + 2] * v[2];
    double vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    return rho * omega[k] * (1.0 + ev / cs2 + ev * ev / (2.0 * cs2 * cs2) - vv / (2.0 * cs2));
}

/* TRT collision, Eq. LBM_collision, with the first-order force term Eq. force_lbm,
 * F_k = omega_k e_k . (rho g) / c_s^2.  Writes fpost (q x n). */
int orc_lbm_collide(int64_t n, int q, const double *e, const double *omega, const int *opp,
                    double tau_p, double tau_m, const double *g, const double *f, double *fpost) {
    const double cs2 = 1.0 / 3.0;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double rho, v[3];
        orc_lbm_moments(q, e, f, n, i, &rho, v);
        for (int k = 0; k < q; ++k) {
            int kb = opp[k];
            double fk = f[(int64_t)k * n + i], fkb = f[(int64_t)kb * n + i];
            double eq = orc_feq(e, omega, k, rho, v), eqb = orc_feq(e, omega, kb, rho, v);
            double fp = 0.5 * (fk + fkb), fm = 0.5 * (fk - fkb);
            double ep = 0.5 * (eq + eqb), em = 0.5 * (eq - eqb);
            double Fk = omega[k] * (e[3 * k] * rho * g[0] + e[3 * k + 1] * rho * g[1] + e[3 * k + 2] * rho * g[2]) / cs2;
            fpost[(int64_t)k * n + i] = fk - (fp - ep) / tau_p - (fm - em) / tau_m + Fk;
        }
    }
    return 0;
}

/* Streaming, Eq. LBM_streaming in the semi-Lagrangian form of the MLBM section:
 * f_k(x_i) = f_k^post at the departure point x_i - dx e_k, interpolated from the
 * stencil of x_i with the weights wk (n x q x n_l; the k = 0 entry is unused since
 * the rest population does not move).  On wall nodes the populations with
 * e_k . n > 0 (departure point inside the solid) are replaced by the opposite
 * streamed population, Eq. interpolated_bounceback_mlbm. */
int orc_lbm_stream(int64_t n, int q, const double *e, const int *opp, const uint8_t *type,
                   const double *nrm, const uint32_t *mask, int n_l, const int32_t *idx, const double *wk,
                   const double *fpost, double *f) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        f[i] = fpost[i];
        for (int k = 1; k < q; ++k) {
            const double *wr = wk + (i * q + k) * n_l;
            double acc = 0.0;
            for (int j = 0; j < n_l; ++j) acc += wr[j] * fpost[(int64_t)k * n + idx[i * n_l + j]];
            f[(int64_t)k * n + i] = acc;
        }
        if (type[i]) {
            const double *nn = nrm + 3 * i;
            for (int k = 1; k < q; ++k) {
                double en = e[3 * k] * nn[0] + e[3 * k + 1] * nn[1] + e[3 * k + 2] * nn[2];
                int unknown = mask ? (int)((mask[i] >> k) & 1u) : en > 0.0;
                if (unknown) f[(int64_t)k * n + i] = f[(int64_t)opp[k] * n + i];
            }
        }
    }
    return 0;
}

/* The streaming step (with bounce-back) of `nrows` selected nodes only: row r is
 * node rows[r], its stencil idx (nrows x n_l, node indices into fpost), weights wk
 * (nrows x q x n_l), type / normal of the selected nodes; fpost (q x n) the whole
 * post-collision field; f (q x nrows) the streamed populations of the rows.  Same
 * arithmetic as orc_lbm_stream, for checking large clouds on a sample. */
int orc_lbm_stream_rows(int64_t nrows, int64_t n, int q, const double *e, const int *opp, const uint8_t *type,
                        const double *nrm, const uint32_t *mask, int n_l, const int32_t *idx, const int64_t *rows,
                        const double *wk, const double *fpost, double *f) {
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < nrows; ++r) {
        f[r] = fpost[rows[r]];
        for (int k = 1; k < q; ++k) {
            const double *wr = wk + (r * q + k) * n_l;
            double acc = 0.0;
            for (int j = 0; j < n_l; ++j) acc += wr[j] * fpost[(int64_t)k * n + idx[r * n_l + j]];
            f[(int64_t)k * nrows + r] = acc;
        }
        if (type[r]) {
            const double *nn = nrm + 3 * r;
            for (int k = 1; k < q; ++k) {
                double en = e[3 * k] * nn[0] + e[3 * k + 1] * nn[1] + e[3 * k + 2] * nn[2];
                int unknown = mask ? (int)((mask[r] >> k) & 1u) : en > 0.0;
                if (unknown) f[(int64_t)k * nrows + r] = f[(int64_t)opp[k] * nrows + r];
            }
        }
    }
    return 0;
}

/* nsteps of the MLBM algorithm of the appendix (COLLIDE over all nodes, then STREAM
 * over all nodes); f (q x n) holds the pre-collision populations in and out. */
int orc_lbm_run(int64_t n, int q, const double *e, const double *omega, const int *opp,
                const uint8_t *type, const double *nrm, const uint32_t *mask, int n_l, const int32_t *idx,
                const double *wk, double tau_p, double tau_m, const double *g, int nsteps, double *f) {
    double *fpost = malloc(sizeof(double) * (size_t)q * n);
    if (!fpost) return -1;
    for (int s = 0; s < nsteps; ++s) {
        orc_lbm_collide(n, q, e, omega, opp, tau_p, tau_m, g, f, fpost);
        orc_lbm_stream(n, q, e, opp, type, nrm, mask, n_l, idx, wk, fpost, f);
    }
    free(fpost);
    return 0;
}

/* Macroscopic rho and v of every node (Eq. macro_var), out (n x 4) = (vx, vy, vz, rho). */
int orc_lbm_macro(int64_t n, int q, const double *e, const double *f, double *out) {
    for (int64_t i = 0; i < n; ++i) {
        double rho, v[3];
        orc_lbm_moments(q, e, f, n, i, &rho, v);
        out[4 * i] = v[0]; out[4 * i + 1] = v[1]; out[4 * i + 2] = v[2]; out[4 * i + 3] = rho;
    }
    return 0;
}

/* ---- stencil application (Eq. operatorApprox) for post-processing -----------
 * out[i*n_ops + o] = sum_j w[(i*n_ops + o)*n_l + j] * u[idx[i*n_l + j]]. */
int orc_apply(int64_t nc, int n_l, const int32_t *idx, int n_ops, const double *w, const double *u,
              double *out) {
    for (int64_t i = 0; i < nc; ++i)
        for (int o = 0; o < n_ops; ++o) {
            double acc = 0.0;
            for (int j = 0; j < n_l; ++j) acc += w[(i * n_ops + o) * n_l + j] * u[idx[i * n_l + j]];
            out[i * n_ops + o] = acc;
        }
    return 0;
}
