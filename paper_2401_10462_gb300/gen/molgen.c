/*
 * Seeded synthetic molecule generators (inputs only; no surface-area arithmetic).
 *
 * Shapes stand in for the paper's protein / RNA / capsid inputs, whose PDB structures
 * and trajectories are not available:
 *   - globule: a self-avoiding chain (bond 1.53 A, non-bonded minimum 2.6 A for |i-j| >= 3,
 *     i,i+2 minimum 2.2 A) confined in a sphere that starts at the radius giving 0.1 atoms/A^3
 *     and grows by 2% whenever placement keeps failing;
 *   - rna: two helical strands (helix radius 20 A, rise 3.4 A, 10 nt per turn, strand 2 shifted
 *     by 180 degrees); each nucleotide is a P atom on the backbone plus a 31-atom chain grown
 *     inward under the same clash rules;
 *   - shell: chains of ~300 atoms filling a spherical shell of thickness 30 A whose outer radius
 *     starts at 150 A and grows by 2% (the fill restarts) until all atoms fit.
 * Radii are drawn from the element mixes of the workloads; every coordinate then gets a
 * uniform jitter in (-1e-6, 1e-6) A.
 *
 * Portability: only integer RNG (splitmix64 seeding, xoshiro256** stream, both from their
 * published definitions) and IEEE +,-,*,/,sqrt are used, compiled with -ffp-contract=off, so
 * the same seed gives the same bits on x86-64 and aarch64.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define PI_D 3.14159265358979323846

/* cube root by Newton iteration (libm cbrt may differ in the last bit between platforms) */
static double cbrt_nr(double a) {
    double x = a > 1.0 ? a / 3.0 : 1.0;
    for (int k = 0; k < 200; ++k) x = x - (x * x * x - a) / (3.0 * x * x);
    return x;
}

typedef struct { uint64_t s[4]; } rng_t;

static uint64_t splitmix64(uint64_t *x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
static void rng_seed(rng_t *r, uint64_t seed) {
    uint64_t x = seed;
    for (int k = 0; k < 4; ++k) r->s[k] = splitmix64(&x);
}
static inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
static uint64_t rng_next(rng_t *r) {
    uint64_t *s = r->s;
    uint64_t res = rotl(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
    s[2] ^= t; s[3] = rotl(s[3], 45);
    return res;
}
static double rng_u01(rng_t *r) { return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0); }
static double rng_sym(rng_t *r) { return 2.0 * rng_u01(r) - 1.0; }
static void rng_dir(rng_t *r, double *v) {
    for (;;) {
        double x = rng_sym(r), y = rng_sym(r), z = rng_sym(r);
        double s = x * x + y * y + z * z;
        if (s > 1e-4 && s <= 1.0) {
            double inv = 1.0 / sqrt(s);
            v[0] = x * inv; v[1] = y * inv; v[2] = z * inv;
            return;
        }
    }
}

/* ---------------------------------------------------------------- clash grid */
#define CELL 2.6
typedef struct {
    double lo[3];
    int dim[3];
    int *head;   /* per cell: first atom, -1 = empty */
    int *next;   /* per atom: next atom in the same cell */
    int *cellof; /* per atom: its cell */
} grid_t;

/* grid over the box [lo, hi] (per axis) padded by one cell */
static int grid_init_box(grid_t *g, const double *lo, const double *hi, int cap) {
    for (int k = 0; k < 3; ++k) {
        g->lo[k] = lo[k] - CELL;
        g->dim[k] = (int)((hi[k] - lo[k] + 2.0 * CELL) / CELL) + 1;
    }
    size_t nc = (size_t)g->dim[0] * (size_t)g->dim[1] * (size_t)g->dim[2];
    if (nc > ((size_t)1 << 31)) return -1;
    g->head = (int *)malloc(nc * sizeof(int));
    g->next = (int *)malloc((size_t)cap * sizeof(int));
    g->cellof = (int *)malloc((size_t)cap * sizeof(int));
    if (!g->head || !g->next || !g->cellof) return -1;
    for (size_t c = 0; c < nc; ++c) g->head[c] = -1;
    return 0;
}
static int grid_init(grid_t *g, double half, int cap) {
    double lo[3] = {-half, -half, -half}, hi[3] = {half, half, half};
    return grid_init_box(g, lo, hi, cap);
}
static void grid_free(grid_t *g) { free(g->head); free(g->next); free(g->cellof); }
static int grid_cell(const grid_t *g, const double *p, int *ijk) {
    for (int k = 0; k < 3; ++k) {
        int c = (int)floor((p[k] - g->lo[k]) / CELL);
        if (c < 0 || c >= g->dim[k]) return -1;
        ijk[k] = c;
    }
    return (int)(((long long)ijk[2] * g->dim[1] + ijk[1]) * g->dim[0] + ijk[0]);
}
static void grid_insert(grid_t *g, const double *p, int id) {
    int ijk[3];
    int c = grid_cell(g, p, ijk);
    g->cellof[id] = c;
    if (c < 0) { g->next[id] = -1; return; }   /* callers only insert points inside the grid */
    g->next[id] = g->head[c];
    g->head[c] = id;
}
/* remove the most recently inserted atom id (it is the head of its cell) */
static void grid_pop(grid_t *g, int id) {
    int c = g->cellof[id];
    if (c < 0) return;
    if (g->head[c] == id) { g->head[c] = g->next[id]; return; }
    int a = g->head[c];
    while (a >= 0 && g->next[a] != id) a = g->next[a];
    if (a >= 0) g->next[a] = g->next[id];
}
/* remove atom id from its cell if it is linked there (no-op otherwise) */
static void grid_pop_if(grid_t *g, int id) {
    int c = g->cellof[id];
    if (c < 0) return;
    for (int a = g->head[c], prev = -1; a >= 0; prev = a, a = g->next[a])
        if (a == id) {
            if (prev < 0) g->head[c] = g->next[a]; else g->next[prev] = g->next[a];
            g->cellof[id] = -1;
            return;
        }
}
/* 1 if p keeps the minimum distances to all placed atoms (ignoring the last bonded ones) */
static int grid_clear(const grid_t *g, const double *xyz, const double *p, int self, int chain_lo) {
    int ijk[3];
    if (grid_cell(g, p, ijk) < 0) return 0;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int x = ijk[0] + dx, y = ijk[1] + dy, z = ijk[2] + dz;
                if (x < 0 || y < 0 || z < 0 || x >= g->dim[0] || y >= g->dim[1] || z >= g->dim[2]) continue;
                for (int a = g->head[((long long)z * g->dim[1] + y) * g->dim[0] + x]; a >= 0; a = g->next[a]) {
                    double ex = p[0] - xyz[3 * a], ey = p[1] - xyz[3 * a + 1], ez = p[2] - xyz[3 * a + 2];
                    double d2 = ex * ex + ey * ey + ez * ez;
                    int sep = self - a; /* chain separation when a is in the same chain */
                    if (a >= chain_lo && sep == 1) continue;
                    double mind = (a >= chain_lo && sep == 2) ? 2.2 : 2.6;
                    if (d2 < mind * mind) return 0;
                }
            }
    return 1;
}

/* ---------------------------------------------------------------- confinement */
enum { CONF_SPHERE = 0, CONF_SHELL = 1, CONF_SLAB = 2 };
typedef struct {
    int kind;
    double r_out, r_in;      /* sphere / shell */
    double axis_r, z_lo, z_hi; /* rna slab around a nucleotide */
} conf_t;
static int conf_ok(const conf_t *c, const double *p) {
    double r2 = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
    if (c->kind == CONF_SPHERE) return r2 <= c->r_out * c->r_out;
    if (c->kind == CONF_SHELL) return r2 <= c->r_out * c->r_out && r2 >= c->r_in * c->r_in;
    double rho2 = p[0] * p[0] + p[1] * p[1];
    return rho2 <= c->axis_r * c->axis_r && p[2] >= c->z_lo && p[2] <= c->z_hi;
}

static const double BOND = 1.53;

/* Grow atoms [start, start+len) of one chain; atom start must already be placed.
 * bias (may be NULL): preferred direction mixed into trial steps. Returns 0 on success. */
static int grow_chain(rng_t *r, grid_t *g, double *xyz, int start, int len, const conf_t *c,
                      const double *bias, int max_fail) {
    int i = start + 1, fails = 0;
    while (i < start + len) {
        int placed = 0;
        for (int t = 0; t < 40 && !placed; ++t) {
            double u[3];
            rng_dir(r, u);
            if (bias) {
                u[0] += 0.3 * bias[0]; u[1] += 0.3 * bias[1]; u[2] += 0.3 * bias[2];
                double s = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
                if (s < 1e-6) continue;
                u[0] /= s; u[1] /= s; u[2] /= s;
            }
            double p[3] = {xyz[3 * (i - 1)] + BOND * u[0], xyz[3 * (i - 1) + 1] + BOND * u[1],
                           xyz[3 * (i - 1) + 2] + BOND * u[2]};
            if (!conf_ok(c, p)) continue;
            if (!grid_clear(g, xyz, p, i, start)) continue;
            xyz[3 * i] = p[0]; xyz[3 * i + 1] = p[1]; xyz[3 * i + 2] = p[2];
            grid_insert(g, p, i);
            placed = 1;
        }
        if (placed) { ++i; continue; }
        if (++fails > max_fail) return -1;
        /* back off further the longer the walk stays stuck */
        int back = 3 + fails / 20;
        if (back > 60) back = 60;
        while (back-- > 0 && i - 1 > start) { --i; grid_pop(g, i); g->cellof[i] = -1; }
    }
    return 0;
}

static void assign_radii(rng_t *r, double *radii, int lo, int n, const double *vals, const double *cum, int k) {
    for (int i = lo; i < lo + n; ++i) {
        double u = rng_u01(r);
        int e = 0;
        while (e < k - 1 && u >= cum[e]) ++e;
        radii[i] = vals[e];
    }
}
static void jitter(rng_t *r, double *xyz, int n) {
    for (int i = 0; i < 3 * n; ++i) xyz[i] += 1e-6 * rng_sym(r);
}

/* protein mix: H 1.2 (50%), C 1.7 (30%), N 1.55 (9%), O 1.52 (10%), S 1.8 (1%) */
static const double PROT_R[5] = {1.2, 1.7, 1.55, 1.52, 1.8};
static const double PROT_C[5] = {0.50, 0.80, 0.89, 0.99, 1.0};
/* nucleotide side atoms: H 40, C 30, N 12, O 16 (renormalised; P sits on the backbone) */
static const double RNA_R[4] = {1.2, 1.7, 1.55, 1.52};
static const double RNA_C[4] = {40.0 / 98, 70.0 / 98, 82.0 / 98, 1.0};

/* Returns achieved confining radius (>0) or -1 on failure. */
double molgen_globule(int n, uint64_t seed, double *xyz, double *radii) {
    if (n <= 0) return 0.0;
    rng_t r;
    rng_seed(&r, seed);
    double rc = cbrt_nr(3.0 * n / (4.0 * PI_D * 0.1));
    for (int attempt = 0; attempt < 200; ++attempt) {
        grid_t g;
        if (grid_init(&g, rc * 1.0001 + 3.0, n) != 0) return -1.0;
        conf_t c = {CONF_SPHERE, rc, 0, 0, 0, 0};
        double u[3];
        rng_dir(&r, u);
        xyz[0] = 0.2 * rc * u[0]; xyz[1] = 0.2 * rc * u[1]; xyz[2] = 0.2 * rc * u[2];
        grid_insert(&g, xyz, 0);
        int ok = grow_chain(&r, &g, xyz, 0, n, &c, NULL, 400 + n / 10) == 0;
        grid_free(&g);
        if (ok) {
            assign_radii(&r, radii, 0, n, PROT_R, PROT_C, 5);
            jitter(&r, xyz, n);
            return rc;
        }
        rc *= 1.02;
    }
    return -1.0;
}

/* Fill a shell with chains of `chain` atoms. Returns achieved outer radius or -1. */
double molgen_shell(int n, uint64_t seed, double r_out0, double thick, int chain, double *xyz, double *radii) {
    if (n <= 0) return 0.0;
    rng_t r;
    rng_seed(&r, seed);
    double ro = r_out0;
    for (int attempt = 0; attempt < 100; ++attempt) {
        grid_t g;
        if (grid_init(&g, ro + 3.0, n) != 0) return -1.0;
        conf_t c = {CONF_SHELL, ro, ro - thick, 0, 0, 0};
        int placed = 0, ok = 1;
        while (placed < n && ok) {
            int len = n - placed < chain ? n - placed : chain;
            int started = 0;
            for (int t = 0; t < 2000 && !started; ++t) {
                double p[3] = {ro * rng_sym(&r), ro * rng_sym(&r), ro * rng_sym(&r)};
                if (!conf_ok(&c, p) || !grid_clear(&g, xyz, p, placed, placed)) continue;
                xyz[3 * placed] = p[0]; xyz[3 * placed + 1] = p[1]; xyz[3 * placed + 2] = p[2];
                grid_insert(&g, p, placed);
                started = 1;
            }
            if (!started) { ok = 0; break; }
            if (grow_chain(&r, &g, xyz, placed, len, &c, NULL, 400) != 0) { ok = 0; break; }
            placed += len;
        }
        grid_free(&g);
        if (ok) {
            assign_radii(&r, radii, 0, n, PROT_R, PROT_C, 5);
            jitter(&r, xyz, n);
            return ro;
        }
        ro *= 1.02;
    }
    return -1.0;
}

/* Double-helix RNA mimic with n atoms (32 per nucleotide; the last one may be partial). */
double molgen_rna(int n, uint64_t seed, double *xyz, double *radii) {
    if (n <= 0) return 0.0;
    rng_t r;
    rng_seed(&r, seed);
    const double helix_r = 20.0, rise = 3.4, per_nt = 32;
    int n_nt = (n + 31) / 32;
    int per_strand = (n_nt + 1) / 2;
    double blo[3] = {-(helix_r + 4.0), -(helix_r + 4.0), -6.0};
    double bhi[3] = {helix_r + 4.0, helix_r + 4.0, rise * per_strand + 6.0};
    grid_t g;
    if (grid_init_box(&g, blo, bhi, n) != 0) return -1.0;
    /* step angle 36 degrees: cos/sin by exact rotation recurrence would drift; use a table of
     * the ten angles computed once from rational constructions via sqrt only. */
    double c36 = (1.0 + sqrt(5.0)) / 4.0;            /* cos 36 */
    double s36 = sqrt(10.0 - 2.0 * sqrt(5.0)) / 4.0; /* sin 36 */
    double ca[10], sa[10];
    ca[0] = 1.0; sa[0] = 0.0;
    for (int k = 1; k < 10; ++k) {
        ca[k] = ca[k - 1] * c36 - sa[k - 1] * s36;
        sa[k] = sa[k - 1] * c36 + ca[k - 1] * s36;
    }
    /* backbone P atoms first (they are >= 12 A apart), then each nucleotide's chain grows
       from its P atom avoiding everything placed so far */
    for (int nt = 0, start = 0; nt < n_nt && start < n; ++nt, start += (int)per_nt) {
        int strand = nt & 1, k = nt >> 1;
        double sgn = strand ? -1.0 : 1.0; /* 180 degree phase shift */
        double p[3] = {sgn * helix_r * ca[k % 10], sgn * helix_r * sa[k % 10], rise * k};
        xyz[3 * start] = p[0]; xyz[3 * start + 1] = p[1]; xyz[3 * start + 2] = p[2];
        grid_insert(&g, p, start);
        radii[start] = 1.9;
    }
    for (int nt = 0, start = 0; nt < n_nt && start < n; ++nt, start += (int)per_nt) {
        int len = n - start < (int)per_nt ? n - start : (int)per_nt;
        if (len <= 1) continue;
        double px = xyz[3 * start], py = xyz[3 * start + 1], pz = xyz[3 * start + 2];
        double inward[3] = {-px / helix_r, -py / helix_r, 0.0};
        int ok_nt = 0;
        /* a crowded nucleotide is regrown; after a few failures its slab widens */
        for (int attempt = 0; attempt < 24 && !ok_nt; ++attempt) {
            double widen = attempt < 4 ? 0.0 : 0.5 * (attempt - 3);
            conf_t c = {CONF_SLAB, 0, 0, helix_r + 2.0 + widen, pz - 4.5 - widen, pz + 4.5 + widen};
            if (grow_chain(&r, &g, xyz, start, len, &c, inward, 200) == 0) ok_nt = 1;
            else for (int id = start + len - 1; id > start; --id) grid_pop_if(&g, id);
        }
        if (!ok_nt) { grid_free(&g); return -1.0; }
        assign_radii(&r, radii, start + 1, len - 1, RNA_R, RNA_C, 4);
    }
    grid_free(&g);
    jitter(&r, xyz, n);
    return helix_r;
}
