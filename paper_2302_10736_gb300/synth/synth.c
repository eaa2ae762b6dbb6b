/*
 * synth.c - seeded synthetic transmission-grid generator.
 *
 * Produces INPUTS only (topology, branch and bus parameters, voltage states,
 * N-1 outage lists, loss weights).  It contains none of the injection or
 * Jacobian arithmetic; both the CPU oracle and the CUDA path consume what it
 * writes.  Plain C99, no platform intrinsics, identical streams on x86-64 and
 * aarch64 for everything that does not go through libm (the Box-Muller and
 * point coordinates use log/cos/sqrt, which can differ by an ulp across libms).
 *
 * Random numbers: xoshiro256** seeded through splitmix64, both as published by
 * Blackman and Vigna ("Scrambled linear pseudorandom number generators", 2018).
 * Every logical stream (topology, parameters, voltages, contingencies, weights)
 * is seeded independently from (seed, stream id).
 *
 * Topology recipe (the paper's MATPOWER cases are not available; these grids
 * stand in for their shape):
 *   - buses are uniform points in the unit square, numbered by a serpentine
 *     sweep over round(sqrt(nb/4)) horizontal bands (regional numbering);
 *   - spanning tree: buses are visited in random order and each joins a
 *     uniformly chosen one of its 3 nearest already-joined buses;
 *   - nl - nb + 1 extra edges: a random bus links to a uniformly chosen one of
 *     its 6 nearest buses; self loops and duplicates are rejected, so the
 *     generated grids have no parallel branches;
 *   - endpoint orientation by coin flip, then a shuffled branch order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SY_PI 3.14159265358979323846

/* ------------------------------------------------------------------ PRNG -- */
typedef struct { uint64_t s[4]; } sy_rng;

static uint64_t sy_splitmix64(uint64_t *x)
{
    uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static void sy_seed(sy_rng *r, uint64_t seed, uint64_t stream)
{
    uint64_t x = (seed << 8) ^ stream;
    for (int i = 0; i < 4; ++i) r->s[i] = sy_splitmix64(&x);
}

static uint64_t sy_rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t sy_next(sy_rng *r)
{
    uint64_t *s = r->s;
    uint64_t out = sy_rotl(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = sy_rotl(s[3], 45);
    return out;
}

/* uniform double in [0, 1) with 53 random bits */
static double sy_u01(sy_rng *r) { return (double)(sy_next(r) >> 11) * (1.0 / 9007199254740992.0); }

static double sy_unif(sy_rng *r, double a, double b) { return a + (b - a) * sy_u01(r); }

/* unbiased integer in [0, n) by rejection of the short final block */
static uint64_t sy_below(sy_rng *r, uint64_t n)
{
    uint64_t lim = (0 - n) % n;
    for (;;) {
        uint64_t v = sy_next(r);
        if (v >= lim) return v % n;
    }
}

/* standard normal pair by the Box-Muller transform */
static void sy_normal2(sy_rng *r, double *z0, double *z1)
{
    double u1 = 1.0 - sy_u01(r); /* (0, 1] */
    double u2 = sy_u01(r);
    double rad = sqrt(-2.0 * log(u1));
    *z0 = rad * cos(2.0 * SY_PI * u2);
    *z1 = rad * sin(2.0 * SY_PI * u2);
}

/* ------------------------------------------------------- spatial buckets -- */
typedef struct {
    int G;          /* cells per side */
    double cs;      /* cell size */
    int *head;      /* G*G, -1 = empty */
    int *next;      /* per point */
} sy_buckets;

static int sy_cell1(double v, int G)
{
    int c = (int)(v * G);
    if (c < 0) c = 0;
    if (c >= G) c = G - 1;
    return c;
}

static int sy_buckets_init(sy_buckets *b, int npts, int G)
{
    b->G = G;
    b->cs = 1.0 / G;
    b->head = (int *)malloc(sizeof(int) * (size_t)G * G);
    b->next = (int *)malloc(sizeof(int) * (size_t)(npts > 0 ? npts : 1));
    if (!b->head || !b->next) return -1;
    for (long i = 0; i < (long)G * G; ++i) b->head[i] = -1;
    return 0;
}

static void sy_buckets_free(sy_buckets *b)
{
    free(b->head);
    free(b->next);
}

static void sy_buckets_insert(sy_buckets *b, int id, double x, double y)
{
    int c = sy_cell1(y, b->G) * b->G + sy_cell1(x, b->G);
    b->next[id] = b->head[c];
    b->head[c] = id;
}

/* k (<= 8) nearest points stored in the buckets, excluding `self`; ties by id.
   Returns how many were found (fewer than k only if the buckets hold fewer). */
static int sy_knn(const sy_buckets *b, const double *px, const double *py, int self, int k,
                  int *best_id, double *best_d)
{
    int G = b->G, cnt = 0;
    double qx = px[self], qy = py[self];
    int cx = sy_cell1(qx, G), cy = sy_cell1(qy, G);
    for (int r = 0; r <= G; ++r) {
        for (int dy = -r; dy <= r; ++dy) {
            int yy = cy + dy;
            if (yy < 0 || yy >= G) continue;
            int step = (dy == -r || dy == r) ? 1 : 2 * r;
            for (int dx = -r; dx <= r; dx += (step > 0 ? step : 1)) {
                int xx = cx + dx;
                if (xx < 0 || xx >= G) continue;
                for (int p = b->head[yy * G + xx]; p >= 0; p = b->next[p]) {
                    if (p == self) continue;
                    double ddx = px[p] - qx, ddy = py[p] - qy;
                    double d = ddx * ddx + ddy * ddy;
                    int pos = cnt;
                    while (pos > 0 && (best_d[pos - 1] > d || (best_d[pos - 1] == d && best_id[pos - 1] > p))) --pos;
                    if (pos >= k) continue;
                    int last = cnt < k ? cnt : k - 1;
                    for (int q = last; q > pos; --q) {
                        best_d[q] = best_d[q - 1];
                        best_id[q] = best_id[q - 1];
                    }
                    best_d[pos] = d;
                    best_id[pos] = p;
                    if (cnt < k) ++cnt;
                }
                if (r == 0) break;
            }
        }
        if (cnt == k) {
            double lim = r * b->cs;
            if (best_d[k - 1] <= lim * lim) break;
        }
    }
    return cnt;
}

/* -------------------------------------------------------------- edge set -- */
typedef struct { uint64_t *key; size_t cap; } sy_set;

static uint64_t sy_key(int a, int b)
{
    int lo = a < b ? a : b, hi = a < b ? b : a;
    return ((uint64_t)(uint32_t)lo << 32) | (uint32_t)hi;
}

static size_t sy_hash(uint64_t k) { return (size_t)((k * 0x9E3779B97F4A7C15ULL) >> 17); }

static int sy_set_init(sy_set *s, size_t n)
{
    size_t cap = 16;
    while (cap < 2 * n + 16) cap <<= 1;
    s->cap = cap;
    s->key = (uint64_t *)malloc(sizeof(uint64_t) * cap);
    if (!s->key) return -1;
    for (size_t i = 0; i < cap; ++i) s->key[i] = UINT64_MAX;
    return 0;
}

/* returns 1 if inserted, 0 if already present */
static int sy_set_add(sy_set *s, uint64_t k)
{
    size_t i = sy_hash(k) & (s->cap - 1);
    while (s->key[i] != UINT64_MAX) {
        if (s->key[i] == k) return 0;
        i = (i + 1) & (s->cap - 1);
    }
    s->key[i] = k;
    return 1;
}

static int sy_set_has(const sy_set *s, uint64_t k)
{
    size_t i = sy_hash(k) & (s->cap - 1);
    while (s->key[i] != UINT64_MAX) {
        if (s->key[i] == k) return 1;
        i = (i + 1) & (s->cap - 1);
    }
    return 0;
}

/* --------------------------------------------------------- serpentine ---- */
typedef struct { int band; double xs; int id; } sy_sk;

static int sy_sk_cmp(const void *a, const void *b)
{
    const sy_sk *p = (const sy_sk *)a, *q = (const sy_sk *)b;
    if (p->band != q->band) return p->band < q->band ? -1 : 1;
    if (p->xs != q->xs) return p->xs < q->xs ? -1 : 1;
    return p->id < q->id ? -1 : (p->id > q->id);
}

/* partial Fisher-Yates: the first m entries of idx[0..n) become a uniform
   m-subset (in random order) */
static void sy_partial_fy(sy_rng *r, int *idx, int n, int m)
{
    for (int i = 0; i < m && i < n; ++i) {
        int j = i + (int)sy_below(r, (uint64_t)(n - i));
        int t = idx[i];
        idx[i] = idx[j];
        idx[j] = t;
    }
}

/* ======================================================== public API ====== */

enum { SY_STREAM_TOPO = 1, SY_STREAM_PARAM = 2, SY_STREAM_VOLT = 3, SY_STREAM_CONT = 4, SY_STREAM_WEIGHT = 5 };

/*
 * Generate one grid.  Arrays are caller-allocated: branch arrays [nl], bus
 * arrays [nb].  Returns 0 on success, -1 on bad sizes (nl < nb-1 or nl larger
 * than the number of distinct bus pairs), -2 on allocation failure.
 *   tx_frac     fraction of branches that are transformers (tap ~ U[0.9,1.1])
 *   shift_max   transformer phase shift ~ U[-shift_max, shift_max] (0: none)
 *   shunt_frac  fraction of buses with a shunt (g_s, b_s ~ U[0, 0.05])
 *   pv_frac     fraction of buses typed PV (bus 0 is the slack)
 */
int sy_grid(int nb, int nl, uint64_t seed, double tx_frac, double shift_max, double shunt_frac,
            double pv_frac, int *from, int *to, double *g, double *b, double *bsh, double *tap,
            double *shift, double *gs, double *bs, int *bustype, double *xcoord, double *ycoord)
{
    if (nb < 1 || nl < nb - 1) return -1;
    if ((double)nl > 0.5 * (double)nb * (double)(nb - 1)) return -1;
    sy_rng rt, rp;
    sy_seed(&rt, seed, SY_STREAM_TOPO);
    sy_seed(&rp, seed, SY_STREAM_PARAM);

    int rc = -2;
    double *x0 = NULL, *y0 = NULL;
    sy_sk *keys = NULL;
    int *perm = NULL, *ef = NULL, *et = NULL, *idx = NULL;
    sy_buckets bj = {0}, ba = {0};
    sy_set es = {0};

    x0 = (double *)malloc(sizeof(double) * nb);
    y0 = (double *)malloc(sizeof(double) * nb);
    keys = (sy_sk *)malloc(sizeof(sy_sk) * nb);
    perm = (int *)malloc(sizeof(int) * nb);
    ef = (int *)malloc(sizeof(int) * (nl > 0 ? nl : 1));
    et = (int *)malloc(sizeof(int) * (nl > 0 ? nl : 1));
    idx = (int *)malloc(sizeof(int) * ((nl > nb ? nl : nb) + 1));
    if (!x0 || !y0 || !keys || !perm || !ef || !et || !idx) goto done;

    /* points and serpentine numbering */
    for (int i = 0; i < nb; ++i) {
        x0[i] = sy_u01(&rt);
        y0[i] = sy_u01(&rt);
    }
    int nrows = (int)llround(sqrt(nb / 4.0));
    if (nrows < 1) nrows = 1;
    for (int i = 0; i < nb; ++i) {
        int band = (int)(y0[i] * nrows);
        if (band >= nrows) band = nrows - 1;
        keys[i].band = band;
        keys[i].xs = (band & 1) ? -x0[i] : x0[i];
        keys[i].id = i;
    }
    qsort(keys, (size_t)nb, sizeof(sy_sk), sy_sk_cmp);
    for (int i = 0; i < nb; ++i) {
        xcoord[i] = x0[keys[i].id];
        ycoord[i] = y0[keys[i].id];
    }

    int G = (int)ceil(sqrt(nb / 2.0));
    if (G < 1) G = 1;
    if (sy_buckets_init(&bj, nb, G) || sy_buckets_init(&ba, nb, G)) goto done;
    if (sy_set_init(&es, (size_t)nl)) goto done;

    /* spanning tree */
    for (int i = 0; i < nb; ++i) perm[i] = i;
    for (int i = nb - 1; i > 0; --i) {
        int j = (int)sy_below(&rt, (uint64_t)(i + 1));
        int t = perm[i];
        perm[i] = perm[j];
        perm[j] = t;
    }
    int ne = 0;
    int bid[8];
    double bd[8];
    sy_buckets_insert(&bj, perm[0], xcoord[perm[0]], ycoord[perm[0]]);
    for (int i = 1; i < nb; ++i) {
        int u = perm[i];
        int cnt = sy_knn(&bj, xcoord, ycoord, u, 3, bid, bd);
        int v = bid[sy_below(&rt, (uint64_t)cnt)];
        ef[ne] = u;
        et[ne] = v;
        sy_set_add(&es, sy_key(u, v));
        ++ne;
        sy_buckets_insert(&bj, u, xcoord[u], ycoord[u]);
    }

    /* extra locality-biased edges */
    for (int i = 0; i < nb; ++i) sy_buckets_insert(&ba, i, xcoord[i], ycoord[i]);
    while (ne < nl) {
        int fails = 0, u = 0, v = 0;
        for (;;) {
            u = (int)sy_below(&rt, (uint64_t)nb);
            if (fails < 256) {
                int cnt = sy_knn(&ba, xcoord, ycoord, u, 6, bid, bd);
                if (cnt == 0) { ++fails; continue; }
                v = bid[sy_below(&rt, (uint64_t)cnt)];
            } else {
                v = (int)sy_below(&rt, (uint64_t)nb);
            }
            if (v != u && !sy_set_has(&es, sy_key(u, v))) break;
            ++fails;
        }
        ef[ne] = u;
        et[ne] = v;
        sy_set_add(&es, sy_key(u, v));
        ++ne;
    }

    /* orientation and branch order */
    for (int l = 0; l < nl; ++l) {
        if (sy_next(&rt) >> 63) {
            int t = ef[l];
            ef[l] = et[l];
            et[l] = t;
        }
    }
    for (int l = 0; l < nl; ++l) idx[l] = l;
    for (int l = nl - 1; l > 0; --l) {
        int j = (int)sy_below(&rt, (uint64_t)(l + 1));
        int t = idx[l];
        idx[l] = idx[j];
        idx[j] = t;
    }
    for (int l = 0; l < nl; ++l) {
        from[l] = ef[idx[l]];
        to[l] = et[idx[l]];
    }

    /* branch parameters */
    for (int l = 0; l < nl; ++l) {
        double r = sy_unif(&rp, 0.001, 0.05);
        double x = sy_unif(&rp, 0.01, 0.3);
        double den = r * r + x * x;
        g[l] = r / den;
        b[l] = -x / den;
        bsh[l] = sy_unif(&rp, 0.0, 0.1);
        tap[l] = 1.0;
        shift[l] = 0.0;
    }
    int ntx = (int)llround(tx_frac * nl);
    for (int l = 0; l < nl; ++l) idx[l] = l;
    sy_partial_fy(&rp, idx, nl, ntx);
    for (int q = 0; q < ntx; ++q) {
        int l = idx[q];
        tap[l] = sy_unif(&rp, 0.9, 1.1);
        if (shift_max > 0.0) shift[l] = sy_unif(&rp, -shift_max, shift_max);
    }

    /* bus shunts and bus types */
    for (int i = 0; i < nb; ++i) {
        gs[i] = 0.0;
        bs[i] = 0.0;
        bustype[i] = 1; /* PQ */
    }
    int nsh = (int)llround(shunt_frac * nb);
    for (int i = 0; i < nb; ++i) idx[i] = i;
    sy_partial_fy(&rp, idx, nb, nsh);
    for (int q = 0; q < nsh; ++q) {
        gs[idx[q]] = sy_unif(&rp, 0.0, 0.05);
        bs[idx[q]] = sy_unif(&rp, 0.0, 0.05);
    }
    bustype[0] = 3; /* slack */
    int npv = (int)llround(pv_frac * nb);
    if (npv > nb - 1) npv = nb - 1;
    for (int i = 0; i < nb - 1; ++i) idx[i] = i + 1;
    sy_partial_fy(&rp, idx, nb - 1, npv);
    for (int q = 0; q < npv; ++q) bustype[idx[q]] = 2; /* PV */
    rc = 0;

done:
    free(x0);
    free(y0);
    free(keys);
    free(perm);
    free(ef);
    free(et);
    free(idx);
    free(es.key);
    if (bj.head) sy_buckets_free(&bj);
    if (ba.head) sy_buckets_free(&ba);
    return rc;
}

/*
 * Voltage states: nscen scenarios laid out [nscen][nb].  |V| ~ U[vlo, vhi],
 * theta ~ N(0, sigma) (Box-Muller), theta of bus `slack` (if >= 0) set to 0.
 * `stream` selects an independent stream so several states can be drawn
 * from one seed (e.g. the state and a second state for target injections).
 */
int sy_voltages(int nb, int nscen, uint64_t seed, int stream, double vlo, double vhi, double sigma,
                int slack, double *vm, double *va)
{
    if (nb < 0 || nscen < 0) return -1;
    sy_rng r;
    sy_seed(&r, seed, (uint64_t)SY_STREAM_VOLT + 16u * (uint64_t)stream);
    size_t n = (size_t)nb * (size_t)nscen;
    for (size_t i = 0; i < n; ++i) vm[i] = sy_unif(&r, vlo, vhi);
    for (size_t i = 0; i < n; i += 2) {
        double z0, z1;
        sy_normal2(&r, &z0, &z1);
        va[i] = sigma * z0;
        if (i + 1 < n) va[i + 1] = sigma * z1;
    }
    if (slack >= 0 && slack < nb)
        for (int s = 0; s < nscen; ++s) va[(size_t)s * nb + slack] = 0.0;
    return 0;
}

/* Bridges of the (multi)graph by Tarjan's low-link method, iterative DFS.
   is_bridge[l] = 1 when removing branch l disconnects its endpoints. */
int sy_bridges(int nb, int nl, const int *from, const int *to, unsigned char *is_bridge)
{
    int rc = -2;
    int *deg = (int *)calloc((size_t)nb + 1, sizeof(int));
    int *adj_v = (int *)malloc(sizeof(int) * (size_t)(2 * nl + 1));
    int *adj_e = (int *)malloc(sizeof(int) * (size_t)(2 * nl + 1));
    int *disc = (int *)malloc(sizeof(int) * (size_t)(nb + 1));
    int *low = (int *)malloc(sizeof(int) * (size_t)(nb + 1));
    int *pe = (int *)malloc(sizeof(int) * (size_t)(nb + 1));
    int *it = (int *)malloc(sizeof(int) * (size_t)(nb + 1));
    int *stk = (int *)malloc(sizeof(int) * (size_t)(nb + 1));
    if (!deg || !adj_v || !adj_e || !disc || !low || !pe || !it || !stk) goto done;
    for (int l = 0; l < nl; ++l) {
        if (from[l] < 0 || from[l] >= nb || to[l] < 0 || to[l] >= nb) { rc = -1; goto done; }
        deg[from[l] + 1]++;
        deg[to[l] + 1]++;
        is_bridge[l] = 0;
    }
    for (int i = 0; i < nb; ++i) deg[i + 1] += deg[i];
    for (int i = 0; i < nb; ++i) it[i] = deg[i];
    for (int l = 0; l < nl; ++l) {
        adj_v[it[from[l]]] = to[l];
        adj_e[it[from[l]]++] = l;
        adj_v[it[to[l]]] = from[l];
        adj_e[it[to[l]]++] = l;
    }
    for (int i = 0; i < nb; ++i) {
        disc[i] = -1;
        it[i] = deg[i];
    }
    int timer = 0;
    for (int root = 0; root < nb; ++root) {
        if (disc[root] >= 0) continue;
        int sp = 0;
        stk[sp++] = root;
        disc[root] = low[root] = timer++;
        pe[root] = -1;
        while (sp > 0) {
            int v = stk[sp - 1];
            if (it[v] < deg[v + 1]) {
                int w = adj_v[it[v]], e = adj_e[it[v]];
                it[v]++;
                if (e == pe[v]) continue;
                if (disc[w] < 0) {
                    pe[w] = e;
                    disc[w] = low[w] = timer++;
                    stk[sp++] = w;
                } else if (disc[w] < low[v]) {
                    low[v] = disc[w];
                }
            } else {
                --sp;
                if (pe[v] >= 0) {
                    int p = stk[sp - 1];
                    if (low[v] < low[p]) low[p] = low[v];
                    if (low[v] > disc[p]) is_bridge[pe[v]] = 1;
                }
            }
        }
    }
    rc = 0;
done:
    free(deg);
    free(adj_v);
    free(adj_e);
    free(disc);
    free(low);
    free(pe);
    free(it);
    free(stk);
    return rc;
}

/* nscen distinct non-bridge branches, uniformly by partial Fisher-Yates.
   Returns -1 if fewer than nscen non-bridge branches exist. */
int sy_outages(int nl, const unsigned char *is_bridge, int nscen, uint64_t seed, int *outage)
{
    int *cand = (int *)malloc(sizeof(int) * (size_t)(nl + 1));
    if (!cand) return -2;
    int nc = 0;
    for (int l = 0; l < nl; ++l)
        if (!is_bridge[l]) cand[nc++] = l;
    if (nc < nscen) {
        free(cand);
        return -1;
    }
    sy_rng r;
    sy_seed(&r, seed, SY_STREAM_CONT);
    sy_partial_fy(&r, cand, nc, nscen);
    for (int s = 0; s < nscen; ++s) outage[s] = cand[s];
    free(cand);
    return 0;
}

/* loss weights w ~ U[lo, hi], [n] each for P and Q */
int sy_weights(int n, uint64_t seed, double lo, double hi, double *wP, double *wQ)
{
    sy_rng r;
    sy_seed(&r, seed, SY_STREAM_WEIGHT);
    for (int i = 0; i < n; ++i) wP[i] = sy_unif(&r, lo, hi);
    for (int i = 0; i < n; ++i) wQ[i] = sy_unif(&r, lo, hi);
    return 0;
}

/* uniform integers in [0, n) (coordinate sampling for finite-difference checks) */
int sy_randint(uint64_t seed, int stream, int count, int n, int *out)
{
    if (n <= 0) return -1;
    sy_rng r;
    sy_seed(&r, seed, 1000u + (uint64_t)stream);
    for (int i = 0; i < count; ++i) out[i] = (int)sy_below(&r, (uint64_t)n);
    return 0;
}
