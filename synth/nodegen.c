/* nodegen.c — seeded synthetic node clouds for periodic simple-cubic sphere cells.
 *
 * Input generation only: nothing here computes any part of the RBF-FD method.
 * Both the CUDA library and the CPU oracle consume the clouds written here, so
 * the two sides see identical inputs.
 *
 * Geometry (periodic unit cell d = 1, one sphere of radius r centred at c) is the
 * case of the paper's case definition section; node spacing follows either a
 * jittered regular grid or a variable-density advancing-front fill in the spirit
 * of the DIVG algorithm described in the meshless-discretisation section (a
 * queue of accepted nodes, candidates on a sphere of radius h(x) around each
 * de-queued node, acceptance when inside the fluid and not closer than h to any
 * node).  Random numbers come from xoshiro256** seeded through SplitMix64
 * (Blackman & Vigna, "Scrambled linear pseudorandom number generators", 2021).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- PRNG: SplitMix64 → xoshiro256** (published definitions) ---------- */
typedef struct { uint64_t s[4]; } sg_rng;

static uint64_t sg_splitmix64(uint64_t *x) {
    uint64_t z = (*x += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}
static uint64_t sg_rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
static void sg_seed(sg_rng *r, uint64_t seed) {
    for (int i = 0; i < 4; ++i) r->s[i] = sg_splitmix64(&seed);
}
static uint64_t sg_next(sg_rng *r) {
    uint64_t *s = r->s;
    uint64_t out = sg_rotl(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
    s[2] ^= t; s[3] = sg_rotl(s[3], 45);
    return out;
}
/* uniform double in [0, 1) with 53 random bits */
static double sg_u01(sg_rng *r) { return (double)(sg_next(r) >> 11) * 0x1.0p-53; }

uint64_t sg_rng_stream(uint64_t seed, int64_t n, uint64_t *out) {
    sg_rng r; sg_seed(&r, seed);
    for (int64_t i = 0; i < n; ++i) out[i] = sg_next(&r);
    return (uint64_t)n;
}

/* ---- geometry helpers ---------------------------------------------------- */
static double sg_wrap01(double x) { x -= floor(x); return x >= 1.0 ? 0.0 : x; }
static double sg_mimg(double d) { return d - rint(d); }
static double sg_sdf(const double c[3], double r, const double x[3]) {
    double dx = sg_mimg(x[0] - c[0]), dy = sg_mimg(x[1] - c[1]), dz = sg_mimg(x[2] - c[2]);
    return sqrt(dx * dx + dy * dy + dz * dz) - r;
}

/* Jittered regular grid: nodes at (i+1/2)h + U[-jit*h, jit*h]^3 (h = 1/n_axis),
 * wrapped into [0,1), dropped when the signed wall distance is < drop*h.
 * Returns the node count (or -1 when cap is too small). */
int64_t sg_jittered_grid(int n_axis, double jit, const double *c, double r, double drop,
                         uint64_t seed, double *out, int64_t cap) {
    sg_rng rng; sg_seed(&rng, seed);
    double h = 1.0 / n_axis;
    int64_t m = 0;
    for (int i = 0; i < n_axis; ++i)
        for (int j = 0; j < n_axis; ++j)
            for (int k = 0; k < n_axis; ++k) {
                double x[3];
                x[0] = (i + 0.5) * h + (2.0 * sg_u01(&rng) - 1.0) * jit * h;
                x[1] = (j + 0.5) * h + (2.0 * sg_u01(&rng) - 1.0) * jit * h;
                x[2] = (k + 0.5) * h + (2.0 * sg_u01(&rng) - 1.0) * jit * h;
                for (int a = 0; a < 3; ++a) x[a] = sg_wrap01(x[a]);
                if (sg_sdf(c, r, x) < drop * h) continue;
                if (m >= cap) return -1;
                memcpy(out + 3 * m, x, sizeof x);
                ++m;
            }
    return m;
}

/* Sphere-surface nodes: a Fibonacci lattice of round(4 pi r^2 / h^2) points on the
 * sphere; points that fall inside a periodic image of the sphere (overlapping grains,
 * r > 1/2) are removed.  Normals are unit vectors pointing out of the solid into the
 * fluid.  Positions are wrapped into [0,1). */
int64_t sg_sphere_surface(const double *c, double r, double h, double *xyz, double *nrm,
                          int64_t cap) {
    const double golden = M_PI * (3.0 - sqrt(5.0));
    int64_t ns = (int64_t)llround(4.0 * M_PI * r * r / (h * h));
    if (ns < 1) ns = 1;
    int64_t m = 0;
    for (int64_t i = 0; i < ns; ++i) {
        double z = 1.0 - (2.0 * i + 1.0) / (double)ns;
        double rho = sqrt(fmax(0.0, 1.0 - z * z));
        double ph = golden * (double)i;
        double n[3] = {rho * cos(ph), rho * sin(ph), z};
        double x[3];
        for (int a = 0; a < 3; ++a) x[a] = sg_wrap01(c[a] + r * n[a]);
        if (sg_sdf(c, r, x) < -1e-9 * r) continue; /* inside another periodic image */
        if (m >= cap) return -1;
        memcpy(xyz + 3 * m, x, sizeof x);
        memcpy(nrm + 3 * m, n, sizeof n);
        ++m;
    }
    return m;
}

/* ---- variable-density advancing-front fill ------------------------------- */
typedef struct {
    int g;            /* cells per axis */
    double cs;        /* cell size */
    int64_t *head;    /* g^3 heads of singly linked lists */
    int64_t *next;    /* per node */
} sg_grid;

static int64_t sg_cell_of(const sg_grid *G, const double x[3]) {
    int i = (int)(x[0] * G->g), j = (int)(x[1] * G->g), k = (int)(x[2] * G->g);
    if (i >= G->g) i = G->g - 1;
    if (j >= G->g) j = G->g - 1;
    if (k >= G->g) k = G->g - 1;
    return ((int64_t)i * G->g + j) * G->g + k;
}

/* Target spacing at wall distance d.  mode 0: linear ramp h_min + (h_max - h_min)
 * min(1, d / shape).  mode 1: the Gaussian of Eq. refinement_function,
 * h_max - exp(-t^2 / (2 shape^2)) (h_max - h_min) with t = d / (sqrt(3)/2 - r) the
 * wall distance over its largest value in the cell (shape = epsilon). */
typedef struct {
    int mode;
    double h_min, h_max, shape, dmax;
} sg_spacing;

static double sg_h_of(const sg_spacing *S, double d) {
    if (S->mode == 1) {
        double t = d / S->dmax;
        return S->h_max - exp(-t * t / (2.0 * S->shape * S->shape)) * (S->h_max - S->h_min);
    }
    double t = d / S->shape;
    if (t > 1.0) t = 1.0;
    if (t < 0.0) t = 0.0;
    return S->h_min + (S->h_max - S->h_min) * t;
}

/* Is there a node within distance `rad` of x (periodic)? */
static int sg_too_close(const sg_grid *G, const double *pts, const double x[3], double rad) {
    int reach = (int)ceil(rad / G->cs);
    if (2 * reach + 1 > G->g) reach = (G->g - 1) / 2;
    int ci = (int)(x[0] * G->g), cj = (int)(x[1] * G->g), ck = (int)(x[2] * G->g);
    double r2 = rad * rad;
    for (int di = -reach; di <= reach; ++di)
        for (int dj = -reach; dj <= reach; ++dj)
            for (int dk = -reach; dk <= reach; ++dk) {
                int i = ((ci + di) % G->g + G->g) % G->g;
                int j = ((cj + dj) % G->g + G->g) % G->g;
                int k = ((ck + dk) % G->g + G->g) % G->g;
                for (int64_t p = G->head[((int64_t)i * G->g + j) * G->g + k]; p >= 0; p = G->next[p]) {
                    double dx = sg_mimg(pts[3 * p] - x[0]);
                    double dy = sg_mimg(pts[3 * p + 1] - x[1]);
                    double dz = sg_mimg(pts[3 * p + 2] - x[2]);
                    if (dx * dx + dy * dy + dz * dz < r2) return 1;
                }
            }
    return 0;
}

/* Fill the fluid part of the periodic cell.  `seed_xyz` (n_seed nodes, e.g. the wall
 * nodes) are placed first and seed the queue.  Spacing h(d) from S, d the wall
 * distance (sg_h_of); a candidate is accepted when its wall
 * distance is > wall_gap*h(d) and no node lies closer than excl*min(h(d), h_p), h_p the
 * spacing at the de-queued node.  n_cand candidates per de-queued node.  Output holds
 * the seeds first, then the fill.  Returns the total count, or -1 when cap is too small. */
static int64_t sg_front(const double *c, double r, const sg_spacing *S, double wall_gap, double excl, int n_cand,
                        uint64_t seed, int64_t n_seed, const double *seed_xyz, double *out, int64_t cap) {
    const double h_min = S->h_min;
    if (cap < n_seed) return -1;
    sg_rng rng; sg_seed(&rng, seed);
    sg_grid G;
    G.g = (int)floor(1.0 / (2.0 * h_min));
    if (G.g < 1) G.g = 1;
    if (G.g > 512) G.g = 512;
    G.cs = 1.0 / G.g;
    int64_t ncell = (int64_t)G.g * G.g * G.g;
    G.head = (int64_t *)malloc(sizeof(int64_t) * ncell);
    G.next = (int64_t *)malloc(sizeof(int64_t) * cap);
    if (!G.head || !G.next) { free(G.head); free(G.next); return -2; }
    for (int64_t i = 0; i < ncell; ++i) G.head[i] = -1;
    int64_t m = 0;
    for (int64_t i = 0; i < n_seed; ++i) {
        for (int a = 0; a < 3; ++a) out[3 * m + a] = sg_wrap01(seed_xyz[3 * i + a]);
        int64_t cl = sg_cell_of(&G, out + 3 * m);
        G.next[m] = G.head[cl]; G.head[cl] = m;
        ++m;
    }
    int64_t qhead = 0; /* queue = nodes [qhead, m) in insertion order */
    while (qhead < m) {
        double p[3] = {out[3 * qhead], out[3 * qhead + 1], out[3 * qhead + 2]};
        ++qhead;
        double hp = sg_h_of(S, fmax(0.0, sg_sdf(c, r, p)));
        for (int t = 0; t < n_cand; ++t) {
            double z = 2.0 * sg_u01(&rng) - 1.0;
            double ph = 2.0 * M_PI * sg_u01(&rng);
            double s = sqrt(fmax(0.0, 1.0 - z * z));
            double x[3] = {p[0] + hp * s * cos(ph), p[1] + hp * s * sin(ph), p[2] + hp * z};
            for (int a = 0; a < 3; ++a) x[a] = sg_wrap01(x[a]);
            double d = sg_sdf(c, r, x);
            if (d <= 0.0) continue;
            double hx = sg_h_of(S, d);
            if (d < wall_gap * hx) continue;
            if (sg_too_close(&G, out, x, excl * fmin(hx, hp))) continue;
            if (m >= cap) { free(G.head); free(G.next); return -1; }
            memcpy(out + 3 * m, x, sizeof x);
            int64_t cl = sg_cell_of(&G, x);
            G.next[m] = G.head[cl]; G.head[cl] = m;
            ++m;
        }
    }
    free(G.head); free(G.next);
    return m;
}

int64_t sg_advancing_front(const double *c, double r, double h_min, double h_max, double ramp,
                           double wall_gap, double excl, int n_cand, uint64_t seed, int64_t n_seed,
                           const double *seed_xyz, double *out, int64_t cap) {
    sg_spacing S = {0, h_min, h_max, ramp, 1.0};
    return sg_front(c, r, &S, wall_gap, excl, n_cand, seed, n_seed, seed_xyz, out, cap);
}

/* As sg_advancing_front with the Gaussian spacing of Eq. refinement_function
 * (shape parameter eps); needs r < sqrt(3)/2. */
int64_t sg_advancing_front_gauss(const double *c, double r, double h_min, double h_max, double eps,
                                 double wall_gap, double excl, int n_cand, uint64_t seed, int64_t n_seed,
                                 const double *seed_xyz, double *out, int64_t cap) {
    if (!(r < 0.5 * sqrt(3.0)) || !(eps > 0.0)) return -3;
    sg_spacing S = {1, h_min, h_max, eps, 0.5 * sqrt(3.0) - r};
    return sg_front(c, r, &S, wall_gap, excl, n_cand, seed, n_seed, seed_xyz, out, cap);
}
