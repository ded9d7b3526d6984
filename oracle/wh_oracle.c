/*
 * CPU ORACLE for the warehouse plan evaluator -- TEST INFRASTRUCTURE ONLY.
 * Plain single-threaded C99; see wh_oracle.h for what it follows and who may
 * use it.  Nothing here is tuned: clarity first, one obvious step at a time.
 */
#include "wh_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define INF64 ((int64_t)1 << 60)

typedef struct { int32_t a; int64_t y; } pick_t;

/* ---------------------------------------------------------------- geometry */

/* back cross-aisle centre depth: Y = W + (L-1)*S */
static int64_t depth_back(const or_layout *g) {
    return (int64_t)g->cross_aisle_width + (int64_t)(g->slots_per_side - 1) * g->slot_pitch;
}

/* Reading of the layout: positive sizes, even cross-aisle width, and the
 * longest S-shape tour 2*x_{A-1} + A*Y below 2^30 so every tour cost fits an
 * int32 with room to spare. */
static int layout_check(const or_layout *g) {
    if (!g || g->n_aisles < 1 || g->slots_per_side < 1 || g->aisle_pitch < 1 ||
        g->slot_pitch < 1 || g->cross_aisle_width < 2 || (g->cross_aisle_width & 1))
        return OR_EINVAL;
    int64_t worst = 2 * (int64_t)(g->n_aisles - 1) * g->aisle_pitch + (int64_t)g->n_aisles * depth_back(g);
    if (worst >= ((int64_t)1 << 30)) return OR_ERANGE;
    return OR_OK;
}

/* location id -> (aisle, depth); loc = (a*2 + side)*L + k, depth = W/2 + k*S */
static int loc_to_pick(const or_layout *g, int32_t loc, pick_t *out) {
    int64_t n_loc = (int64_t)g->n_aisles * 2 * g->slots_per_side;
    if (loc < 0 || loc >= n_loc) return OR_ERANGE;
    int32_t a = loc / (2 * g->slots_per_side);
    int32_t k = loc % g->slots_per_side;
    out->a = a;
    out->y = g->cross_aisle_width / 2 + (int64_t)k * g->slot_pitch;
    return OR_OK;
}

int64_t or_dist(const or_layout *g, int32_t a1, int32_t y1, int32_t a2, int32_t y2) {
    int64_t Y = depth_back(g);
    if (a1 == a2) return y1 > y2 ? (int64_t)y1 - y2 : (int64_t)y2 - y1;
    int64_t dx = (int64_t)(a1 > a2 ? a1 - a2 : a2 - a1) * g->aisle_pitch;
    int64_t via_front = (int64_t)y1 + y2;
    int64_t via_back = 2 * Y - y1 - y2;
    return dx + (via_front < via_back ? via_front : via_back);
}

static int cmp_pick(const void *p, const void *q) {
    const pick_t *u = (const pick_t *)p, *v = (const pick_t *)q;
    if (u->a != v->a) return u->a < v->a ? -1 : 1;
    return u->y < v->y ? -1 : (u->y > v->y);
}

/* The tour's pick set: decode, sort by (aisle, depth), drop duplicates.
 * Returns the number of distinct picks or an error. */
static int32_t pick_set(const or_layout *g, const int32_t *locs, int32_t n, pick_t **out) {
    *out = NULL;
    if (n < 0) return OR_EINVAL;
    if (n == 0) return 0;
    pick_t *p = (pick_t *)malloc(sizeof(pick_t) * (size_t)n);
    if (!p) return OR_ENOMEM;
    for (int32_t i = 0; i < n; ++i) {
        if (loc_to_pick(g, locs[i], &p[i]) != OR_OK) { free(p); return OR_ERANGE; }
    }
    qsort(p, (size_t)n, sizeof(pick_t), cmp_pick);
    int32_t m = 0;
    for (int32_t i = 0; i < n; ++i)
        if (m == 0 || p[i].a != p[m - 1].a || p[i].y != p[m - 1].y) p[m++] = p[i];
    *out = p;
    return m;
}

/* ----------------------------------------------------------------- S-shape */

/* S-shape route, simulated as a walk (routing rule: the S-shape heuristic).
 * The picker leaves the depot along the front cross-aisle, enters the pick
 * aisles from left to right and traverses each one completely, alternately
 * front-to-back and back-to-front, moving between consecutive pick aisles along
 * whichever cross-aisle it stands on.  When the number of pick aisles is odd,
 * the last one is entered from the front, walked up to its deepest pick and
 * left again at the front.  The picker then walks back to the depot along the
 * front cross-aisle.  Aisles without picks are never entered. */
int64_t or_sshape_tour(const or_layout *g, const int32_t *locs, int32_t n) {
    int rc = layout_check(g);
    if (rc != OR_OK) return rc;
    pick_t *p;
    int32_t m = pick_set(g, locs, n, &p);
    if (m < 0) return m;
    if (m == 0) return 0;
    int64_t Y = depth_back(g);
    /* the pick aisles, left to right, with the deepest pick of each */
    int32_t *aisle = (int32_t *)malloc(sizeof(int32_t) * (size_t)m);
    int64_t *deep = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
    int32_t na = 0;
    for (int32_t i = 0; i < m; ++i) {
        if (na == 0 || aisle[na - 1] != p[i].a) { aisle[na] = p[i].a; deep[na] = p[i].y; ++na; }
        else if (p[i].y > deep[na - 1]) deep[na - 1] = p[i].y;
    }
    int64_t walked = 0;
    int64_t x = 0;       /* horizontal position of the picker */
    int64_t depth = 0;   /* 0 = on the front cross-aisle, Y = on the back one */
    for (int32_t q = 0; q < na; ++q) {
        int64_t xa = (int64_t)aisle[q] * g->aisle_pitch;
        walked += xa > x ? xa - x : x - xa;  /* along the current cross-aisle */
        x = xa;
        if (q == na - 1 && (na % 2) == 1) {
            /* odd number of pick aisles: the picker is at the front here */
            walked += 2 * deep[q];
        } else {
            walked += Y;                     /* full traversal of the aisle */
            depth = (depth == 0) ? Y : 0;
        }
    }
    walked += x;                             /* back along the front to the depot */
    free(aisle);
    free(deep);
    free(p);
    (void)depth;
    return walked;
}

/* ----------------------------------------------------- Ratliff-Rosenthal DP */

/* Degree label of an aisle end vertex in a partial tour subgraph. */
enum { D0 = 0, DE = 1, DU = 2 }; /* not in the subgraph / even degree / odd degree */

/* The seven equivalence classes (deg a_j, deg b_j, number of components):
 * (U,U,1C) (0,E,1C) (E,0,1C) (E,E,1C) (E,E,2C) (0,0,0C) (0,0,1C). */
typedef struct { int da, db, nc; } cls_t;
static const cls_t CLASSES[7] = {
    {DU, DU, 1}, {D0, DE, 1}, {DE, D0, 1}, {DE, DE, 1}, {DE, DE, 2}, {D0, D0, 0}, {D0, D0, 1}};
enum { C_UU1 = 0, C_0E1, C_E01, C_EE1, C_EE2, C_000, C_001 };

/* A component of a partial subgraph, described by which of the two current
 * aisle ends it contains.  A component containing neither is closed. */
typedef struct { int has_a, has_b; } comp_t;

typedef struct {
    int in_a, in_b;     /* vertex belongs to the subgraph */
    int odd_a, odd_b;   /* degree parity */
    int n;              /* number of components */
    comp_t c[4];
} graph_state_t;

static graph_state_t state_of_class(int k) {
    graph_state_t s;
    memset(&s, 0, sizeof(s));
    cls_t c = CLASSES[k];
    s.in_a = c.da != D0; s.odd_a = c.da == DU;
    s.in_b = c.db != D0; s.odd_b = c.db == DU;
    if (c.nc == 0) { s.n = 0; }
    else if (c.nc == 2) { s.n = 2; s.c[0].has_a = 1; s.c[1].has_b = 1; }
    else { s.n = 1; s.c[0].has_a = s.in_a; s.c[0].has_b = s.in_b; }
    return s;
}

/* merge components that share an aisle end */
static void merge_components(graph_state_t *s) {
    int changed = 1;
    while (changed) {
        changed = 0;
        for (int i = 0; i < s->n && !changed; ++i)
            for (int j = i + 1; j < s->n && !changed; ++j)
                if ((s->c[i].has_a && s->c[j].has_a) || (s->c[i].has_b && s->c[j].has_b)) {
                    s->c[i].has_a |= s->c[j].has_a;
                    s->c[i].has_b |= s->c[j].has_b;
                    s->c[j] = s->c[s->n - 1];
                    --s->n;
                    changed = 1;
                }
    }
}

/* Classify a state; -1 when it is not one of the seven classes (for instance
 * a closed component beside an open one, which can never become one tour). */
static int class_of_state(const graph_state_t *s) {
    int open = 0, closed = 0;
    for (int i = 0; i < s->n; ++i) {
        if (s->c[i].has_a || s->c[i].has_b) ++open; else ++closed;
    }
    if (closed > 0 && (open > 0 || closed > 1)) return -1;
    int da = s->in_a ? (s->odd_a ? DU : DE) : D0;
    int db = s->in_b ? (s->odd_b ? DU : DE) : D0;
    int nc = s->n;
    if (closed == 1) { da = D0; db = D0; }
    for (int k = 0; k < 7; ++k) {
        if (CLASSES[k].da != da || CLASSES[k].db != db || CLASSES[k].nc != nc) continue;
        if (k == C_EE1 || k == C_UU1) {
            if (!(s->c[0].has_a && s->c[0].has_b)) return -1;
        }
        return k;
    }
    return -1;
}

/* Vertical configurations of one aisle (its picks p_1 <= ... <= p_k):
 *   full traverse        cost Y,         +1 at a_j and b_j, one piece a..b
 *   double traverse      cost 2Y,        +2 / +2, one piece a..b
 *   largest gap left out cost 2(Y-g),    +2 / +2, a piece at a and one at b
 *   from the back only   cost 2(Y-p_1),  0 / +2, a piece at b
 *   from the front only  cost 2 p_k,     +2 / 0, a piece at a
 *   none                 cost 0          (only when the aisle has no pick)
 * with g the largest gap between consecutive members of {0, p_1..p_k, Y}. */
typedef struct { int64_t cost; int da, db; int npieces; comp_t piece[2]; } vopt_t;

static int vertical_options(const int64_t *p, int32_t k, int64_t Y, vopt_t *o) {
    if (k == 0) {
        o[0].cost = 0; o[0].da = 0; o[0].db = 0; o[0].npieces = 0;
        return 1;
    }
    int64_t g = p[0];
    for (int32_t i = 1; i < k; ++i) if (p[i] - p[i - 1] > g) g = p[i] - p[i - 1];
    if (Y - p[k - 1] > g) g = Y - p[k - 1];
    comp_t ab = {1, 1}, a = {1, 0}, b = {0, 1};
    o[0] = (vopt_t){Y, 1, 1, 1, {ab, ab}};
    o[1] = (vopt_t){2 * Y, 2, 2, 1, {ab, ab}};
    o[2] = (vopt_t){2 * (Y - g), 2, 2, 2, {a, b}};
    o[3] = (vopt_t){2 * (Y - p[0]), 0, 2, 1, {b, b}};
    o[4] = (vopt_t){2 * p[k - 1], 2, 0, 1, {a, a}};
    return 5;
}

static int apply_vertical(int cls, const vopt_t *v) {
    graph_state_t s = state_of_class(cls);
    if (v->npieces == 0) return cls;
    for (int i = 0; i < v->npieces; ++i) s.c[s.n++] = v->piece[i];
    if (v->da) { s.in_a = 1; s.odd_a ^= (v->da & 1); }
    if (v->db) { s.in_b = 1; s.odd_b ^= (v->db & 1); }
    merge_components(&s);
    return class_of_state(&s);
}

/* Horizontal edges between aisle j-1 and j: xa copies of a_{j-1}a_j and xb of
 * b_{j-1}b_j, from the five combinations (1,1) (2,0) (0,2) (2,2) (0,0).  After
 * this step a_{j-1} and b_{j-1} get no more edges, so their degrees must be
 * even; a vertex outside the subgraph gets no edge. */
static int apply_horizontal(int cls, int xa, int xb) {
    graph_state_t s = state_of_class(cls);
    if ((s.odd_a + xa) % 2 != 0 || (s.odd_b + xb) % 2 != 0) return -1;
    if ((!s.in_a && xa > 0) || (!s.in_b && xb > 0)) return -1;
    graph_state_t t;
    memset(&t, 0, sizeof(t));
    t.in_a = xa > 0; t.odd_a = xa & 1;
    t.in_b = xb > 0; t.odd_b = xb & 1;
    t.n = s.n;
    for (int i = 0; i < s.n; ++i) {
        t.c[i].has_a = s.c[i].has_a && xa > 0;
        t.c[i].has_b = s.c[i].has_b && xb > 0;
    }
    return class_of_state(&t);
}

/* Optimal tour length by the Ratliff-Rosenthal dynamic programme over the
 * aisles 0..r (r = rightmost aisle with a pick).  The depot is a required
 * pick at depth 0 of aisle 0, so aisle 0 always has a pick; the DP starts in
 * class (0,0,0C) and the answer is the cheapest class after aisle r that is a
 * single component with all degrees even. */
int64_t or_rr_tour(const or_layout *g, const int32_t *locs, int32_t n) {
    int rc = layout_check(g);
    if (rc != OR_OK) return rc;
    pick_t *p;
    int32_t m = pick_set(g, locs, n, &p);
    if (m < 0) return m;
    if (m == 0) return 0;
    int64_t Y = depth_back(g);
    int32_t r = p[m - 1].a;
    int64_t *depths = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m + 1));
    int64_t cost[7], next[7];
    for (int k = 0; k < 7; ++k) cost[k] = INF64;
    cost[C_000] = 0;
    static const int HX[5][2] = {{1, 1}, {2, 0}, {0, 2}, {2, 2}, {0, 0}};
    int32_t i = 0;
    for (int32_t j = 0; j <= r; ++j) {
        if (j > 0) {
            for (int k = 0; k < 7; ++k) next[k] = INF64;
            for (int k = 0; k < 7; ++k) {
                if (cost[k] >= INF64) continue;
                for (int h = 0; h < 5; ++h) {
                    int t = apply_horizontal(k, HX[h][0], HX[h][1]);
                    if (t < 0) continue;
                    int64_t c = cost[k] + (int64_t)(HX[h][0] + HX[h][1]) * g->aisle_pitch;
                    if (c < next[t]) next[t] = c;
                }
            }
            memcpy(cost, next, sizeof(cost));
        }
        /* the picks of aisle j, ascending (the depot counts as one in aisle 0) */
        int32_t k = 0;
        if (j == 0) depths[k++] = 0;
        while (i < m && p[i].a == j) depths[k++] = p[i++].y;
        vopt_t opt[5];
        int no = vertical_options(depths, k, Y, opt);
        for (int q = 0; q < 7; ++q) next[q] = INF64;
        for (int q = 0; q < 7; ++q) {
            if (cost[q] >= INF64) continue;
            for (int v = 0; v < no; ++v) {
                int t = apply_vertical(q, &opt[v]);
                if (t < 0) continue;
                int64_t c = cost[q] + opt[v].cost;
                if (c < next[t]) next[t] = c;
            }
        }
        memcpy(cost, next, sizeof(cost));
    }
    int64_t best = INF64;
    const int finals[4] = {C_EE1, C_E01, C_0E1, C_001};
    for (int f = 0; f < 4; ++f) if (cost[finals[f]] < best) best = cost[finals[f]];
    free(depths);
    free(p);
    return best;
}

/* ------------------------------------------------------ exact small tours */

/* Held-Karp over {depot} + distinct picks with the grid distance. */
int64_t or_heldkarp_tour(const or_layout *g, const int32_t *locs, int32_t n) {
    int rc = layout_check(g);
    if (rc != OR_OK) return rc;
    pick_t *p;
    int32_t m = pick_set(g, locs, n, &p);
    if (m < 0) return m;
    if (m == 0) return 0;
    if (m > 16) { free(p); return OR_ERANGE; }
    int64_t d0[16], d[16][16];
    for (int i = 0; i < m; ++i) {
        d0[i] = or_dist(g, 0, 0, p[i].a, (int32_t)p[i].y);
        for (int j = 0; j < m; ++j) d[i][j] = or_dist(g, p[i].a, (int32_t)p[i].y, p[j].a, (int32_t)p[j].y);
    }
    size_t nsub = (size_t)1 << m;
    int64_t *best = (int64_t *)malloc(sizeof(int64_t) * nsub * (size_t)m);
    if (!best) { free(p); return OR_ENOMEM; }
    for (size_t s = 0; s < nsub * (size_t)m; ++s) best[s] = INF64;
    /* best[S][last]: shortest path from the depot through exactly S ending at last */
    for (int i = 0; i < m; ++i) best[((size_t)1 << i) * m + i] = d0[i];
    for (size_t s = 1; s < nsub; ++s)
        for (int last = 0; last < m; ++last) {
            int64_t b = best[s * m + last];
            if (!(s >> last & 1) || b >= INF64) continue;
            for (int nx = 0; nx < m; ++nx) {
                if (s >> nx & 1) continue;
                size_t t = s | ((size_t)1 << nx);
                int64_t c = b + d[last][nx];
                if (c < best[t * m + nx]) best[t * m + nx] = c;
            }
        }
    int64_t ans = INF64;
    for (int last = 0; last < m; ++last) {
        int64_t c = best[(nsub - 1) * m + last] + d0[last];
        if (c < ans) ans = c;
    }
    free(best);
    free(p);
    return ans;
}

/* Every permutation of the picking sequence (the paper's own statement of how
 * the minimum route is found), lexicographic enumeration. */
int64_t or_permutation_tour(const or_layout *g, const int32_t *locs, int32_t n) {
    int rc = layout_check(g);
    if (rc != OR_OK) return rc;
    pick_t *p;
    int32_t m = pick_set(g, locs, n, &p);
    if (m < 0) return m;
    if (m == 0) return 0;
    if (m > 10) { free(p); return OR_ERANGE; }
    int idx[10];
    for (int i = 0; i < m; ++i) idx[i] = i;
    int64_t ans = INF64;
    for (;;) {
        int64_t c = or_dist(g, 0, 0, p[idx[0]].a, (int32_t)p[idx[0]].y);
        for (int i = 0; i + 1 < m; ++i)
            c += or_dist(g, p[idx[i]].a, (int32_t)p[idx[i]].y, p[idx[i + 1]].a, (int32_t)p[idx[i + 1]].y);
        c += or_dist(g, p[idx[m - 1]].a, (int32_t)p[idx[m - 1]].y, 0, 0);
        if (c < ans) ans = c;
        /* next permutation */
        int i = m - 2;
        while (i >= 0 && idx[i] > idx[i + 1]) --i;
        if (i < 0) break;
        int j = m - 1;
        while (idx[j] < idx[i]) --j;
        int t = idx[i]; idx[i] = idx[j]; idx[j] = t;
        for (int a = i + 1, b = m - 1; a < b; ++a, --b) { t = idx[a]; idx[a] = idx[b]; idx[b] = t; }
    }
    free(p);
    return ans;
}

/* ------------------------------------------------------------------- plans */

/* Plan cost = sum over the plan's tours of the tour length (Eq. 2, sum d_i),
 * per routing rule, in int64.  A tour's picks are the locations of the SKUs of
 * all lines of all its orders. */
int or_eval_plans(const or_layout *g, int32_t n_orders, const int32_t *order_off,
                  const int32_t *line_sku, int32_t n_sku, const int32_t *slot_map,
                  int64_t slot_map_stride, int32_t n_plans, const int32_t *plan_tour_off,
                  const int32_t *tour_off, const int32_t *order_seq, int32_t *tour_s,
                  int32_t *tour_rr, int64_t *plan_s, int64_t *plan_rr) {
    int rc = layout_check(g);
    if (rc != OR_OK) return rc;
    if (n_orders < 0 || n_plans < 0 || n_sku < 0 || slot_map_stride < 0) return OR_EINVAL;
    int64_t cap = 64;
    int32_t *buf = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    if (!buf) return OR_ENOMEM;
    for (int32_t pl = 0; pl < n_plans; ++pl) {
        const int32_t *smap = slot_map + (int64_t)pl * slot_map_stride;
        int64_t sum_s = 0, sum_rr = 0;
        if (plan_tour_off[pl + 1] < plan_tour_off[pl]) { free(buf); return OR_EINVAL; }
        for (int32_t t = plan_tour_off[pl]; t < plan_tour_off[pl + 1]; ++t) {
            if (tour_off[t + 1] < tour_off[t]) { free(buf); return OR_EINVAL; }
            int64_t nl = 0;
            for (int32_t q = tour_off[t]; q < tour_off[t + 1]; ++q) {
                int32_t o = order_seq[q];
                if (o < 0 || o >= n_orders) { free(buf); return OR_ERANGE; }
                for (int32_t l = order_off[o]; l < order_off[o + 1]; ++l) {
                    int32_t sku = line_sku[l];
                    if (sku < 0 || sku >= n_sku) { free(buf); return OR_ERANGE; }
                    if (nl == cap) {
                        cap *= 2;
                        int32_t *nb = (int32_t *)realloc(buf, sizeof(int32_t) * (size_t)cap);
                        if (!nb) { free(buf); return OR_ENOMEM; }
                        buf = nb;
                    }
                    buf[nl++] = smap[sku];
                }
            }
            int64_t cs = or_sshape_tour(g, buf, (int32_t)nl);
            int64_t cr = or_rr_tour(g, buf, (int32_t)nl);
            if (cs < 0 || cr < 0) { free(buf); return (int)(cs < 0 ? cs : cr); }
            if (tour_s) tour_s[t] = (int32_t)cs;
            if (tour_rr) tour_rr[t] = (int32_t)cr;
            sum_s += cs;
            sum_rr += cr;
        }
        if (plan_s) plan_s[pl] = sum_s;
        if (plan_rr) plan_rr[pl] = sum_rr;
    }
    free(buf);
    return OR_OK;
}

/* ------------------------------------------------------------------- moves */

/* One plan held as separate order lists per tour, so a move can be applied
 * to a copy by editing lists. */
typedef struct {
    int32_t n_tours;
    int32_t *len;      /* orders per tour */
    int32_t *cap;      /* capacity of each list */
    int32_t **orders;  /* order ids per tour */
} plan_copy_t;

static void plan_free(plan_copy_t *c) {
    for (int32_t t = 0; t < c->n_tours; ++t) free(c->orders[t]);
    free(c->orders);
    free(c->len);
    free(c->cap);
}

static int plan_load(plan_copy_t *c, int32_t p, const int32_t *plan_tour_off, const int32_t *tour_off,
                     const int32_t *order_seq) {
    int32_t t0 = plan_tour_off[p], t1 = plan_tour_off[p + 1];
    c->n_tours = t1 - t0;
    c->len = (int32_t *)calloc((size_t)c->n_tours + 1, sizeof(int32_t));
    c->cap = (int32_t *)calloc((size_t)c->n_tours + 1, sizeof(int32_t));
    c->orders = (int32_t **)calloc((size_t)c->n_tours + 1, sizeof(int32_t *));
    if (!c->len || !c->cap || !c->orders) return OR_ENOMEM;
    for (int32_t t = 0; t < c->n_tours; ++t) {
        int32_t q0 = tour_off[t0 + t], q1 = tour_off[t0 + t + 1];
        c->len[t] = q1 - q0;
        c->cap[t] = q1 - q0 + 1;
        c->orders[t] = (int32_t *)malloc(sizeof(int32_t) * (size_t)c->cap[t]);
        if (!c->orders[t]) return OR_ENOMEM;
        memcpy(c->orders[t], order_seq + q0, sizeof(int32_t) * (size_t)(q1 - q0));
    }
    return OR_OK;
}

/* index of the tour holding order o, or -1 */
static int32_t plan_find(const plan_copy_t *c, int32_t o, int32_t *pos) {
    for (int32_t t = 0; t < c->n_tours; ++t)
        for (int32_t i = 0; i < c->len[t]; ++i)
            if (c->orders[t][i] == o) { *pos = i; return t; }
    return -1;
}

static int32_t tour_line_count(const plan_copy_t *c, int32_t t, const int32_t *order_off) {
    int32_t n = 0;
    for (int32_t i = 0; i < c->len[t]; ++i) n += order_off[c->orders[t][i] + 1] - order_off[c->orders[t][i]];
    return n;
}

/* Sum of both rules over every tour of the plan copy under slotting smap. */
static int plan_cost(const or_layout *g, const plan_copy_t *c, const int32_t *order_off, const int32_t *line_sku,
                     const int32_t *smap, int64_t *sum_s, int64_t *sum_rr) {
    *sum_s = 0;
    *sum_rr = 0;
    for (int32_t t = 0; t < c->n_tours; ++t) {
        int32_t n = tour_line_count(c, t, order_off);
        int32_t *locs = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
        if (!locs) return OR_ENOMEM;
        int32_t k = 0;
        for (int32_t i = 0; i < c->len[t]; ++i) {
            int32_t o = c->orders[t][i];
            for (int32_t l = order_off[o]; l < order_off[o + 1]; ++l) locs[k++] = smap[line_sku[l]];
        }
        int64_t cs = or_sshape_tour(g, locs, n), cr = or_rr_tour(g, locs, n);
        free(locs);
        if (cs < 0 || cr < 0) return (int)(cs < 0 ? cs : cr);
        *sum_s += cs;
        *sum_rr += cr;
    }
    return OR_OK;
}

int or_eval_moves(const or_layout *g, int32_t n_orders, const int32_t *order_off, const int32_t *line_sku,
                  int32_t n_sku, const int32_t *slot_map, int64_t slot_map_stride, int32_t n_plans,
                  const int32_t *plan_tour_off, const int32_t *tour_off, const int32_t *order_seq,
                  const int32_t *moves, int32_t n_moves, int32_t max_orders, int32_t max_lines, int64_t *delta,
                  int32_t *status) {
    int rc = layout_check(g);
    if (rc != OR_OK) return rc;
    int32_t *smap_copy = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_sku > 0 ? n_sku : 1));
    if (!smap_copy) return OR_ENOMEM;
    for (int32_t m = 0; m < n_moves; ++m) {
        const int32_t type = moves[4 * m], a = moves[4 * m + 1], b = moves[4 * m + 2], p = moves[4 * m + 3];
        delta[2 * m] = delta[2 * m + 1] = 0;
        status[m] = 3;
        if (p < 0 || p >= n_plans) continue;
        const int32_t *smap = slot_map + (int64_t)p * slot_map_stride;
        plan_copy_t c;
        memset(&c, 0, sizeof(c));
        rc = plan_load(&c, p, plan_tour_off, tour_off, order_seq);
        if (rc != OR_OK) { plan_free(&c); free(smap_copy); return rc; }
        int64_t before_s, before_rr;
        rc = plan_cost(g, &c, order_off, line_sku, smap, &before_s, &before_rr);
        if (rc != OR_OK) { plan_free(&c); free(smap_copy); return rc; }
        const int32_t *after_map = smap;
        int32_t st = 0;
        if (type == 0 || type == 1) {
            int32_t ia = 0, ib = 0;
            int32_t ta = (a >= 0 && a < n_orders) ? plan_find(&c, a, &ia) : -1;
            if (ta < 0) st = 3;
            else if (type == 0) {
                int32_t tb = (b >= 0 && b < n_orders) ? plan_find(&c, b, &ib) : -1;
                if (tb < 0) st = 3;
                else if (ta == tb) st = 2;
                else {
                    c.orders[ta][ia] = b;
                    c.orders[tb][ib] = a;
                    if (max_lines > 0 && (tour_line_count(&c, ta, order_off) > max_lines ||
                                          tour_line_count(&c, tb, order_off) > max_lines))
                        st = 1;
                }
            } else {
                if (b < 0 || b >= c.n_tours) st = 3;
                else if (b == ta) st = 2;
                else {
                    /* remove a from ta, append to b */
                    for (int32_t i = ia; i + 1 < c.len[ta]; ++i) c.orders[ta][i] = c.orders[ta][i + 1];
                    --c.len[ta];
                    if (c.len[b] == c.cap[b]) {
                        int32_t *nb = (int32_t *)realloc(c.orders[b], sizeof(int32_t) * (size_t)(c.cap[b] + 1));
                        if (!nb) { plan_free(&c); free(smap_copy); return OR_ENOMEM; }
                        c.orders[b] = nb;
                        ++c.cap[b];
                    }
                    c.orders[b][c.len[b]++] = a;
                    if ((max_orders > 0 && c.len[b] > max_orders) ||
                        (max_lines > 0 && tour_line_count(&c, b, order_off) > max_lines))
                        st = 1;
                }
            }
        } else if (type == 2) {
            if (slot_map_stride == 0 || a < 0 || a >= n_sku || b < 0 || b >= n_sku) st = 3;
            else if (a == b) st = 2;
            else {
                memcpy(smap_copy, smap, sizeof(int32_t) * (size_t)n_sku);
                int32_t tmp = smap_copy[a];
                smap_copy[a] = smap_copy[b];
                smap_copy[b] = tmp;
                after_map = smap_copy;
            }
        } else if (type == 3) {
            /* relocate SKU a to location b, which no SKU of the plan holds */
            const int64_t n_loc = (int64_t)g->n_aisles * 2 * g->slots_per_side;
            if (slot_map_stride == 0 || a < 0 || a >= n_sku || b < 0 || b >= n_loc) st = 3;
            else if (smap[a] == b) st = 2;
            else {
                for (int32_t s = 0; s < n_sku; ++s)
                    if (smap[s] == b) { st = 3; break; }
                if (st == 0) {
                    memcpy(smap_copy, smap, sizeof(int32_t) * (size_t)n_sku);
                    smap_copy[a] = b;
                    after_map = smap_copy;
                }
            }
        } else {
            st = 3;
        }
        status[m] = st;
        if (st == 0) {
            int64_t after_s, after_rr;
            rc = plan_cost(g, &c, order_off, line_sku, after_map, &after_s, &after_rr);
            if (rc != OR_OK) { plan_free(&c); free(smap_copy); return rc; }
            delta[2 * m] = after_s - before_s;
            delta[2 * m + 1] = after_rr - before_rr;
        }
        plan_free(&c);
    }
    free(smap_copy);
    return OR_OK;
}

/* ---------------------------------------------------------- local search */

int or_ls_step(const or_layout *g, int32_t n_orders, const int32_t *order_off, const int32_t *line_sku,
               int32_t n_sku, int32_t *slot_map, int64_t slot_map_stride, int32_t n_plans,
               const int32_t *plan_tour_off, int32_t *tour_off, int32_t *order_seq, const int32_t *moves,
               int32_t moves_per_plan, int32_t max_orders, int32_t max_lines, int32_t *applied) {
    const int32_t M = moves_per_plan;
    int64_t *delta = (int64_t *)malloc(sizeof(int64_t) * 2 * (size_t)(M > 0 ? M : 1));
    int32_t *status = (int32_t *)malloc(sizeof(int32_t) * (size_t)(M > 0 ? M : 1));
    if (!delta || !status) { free(delta); free(status); return OR_ENOMEM; }
    for (int32_t p = 0; p < n_plans; ++p) {
        applied[p] = -1;
        const int32_t *mv = moves + (int64_t)p * M * 4;
        /* every move of this plan is scored against the plan as it is now */
        int rc = or_eval_moves(g, n_orders, order_off, line_sku, n_sku, slot_map, slot_map_stride, n_plans,
                               plan_tour_off, tour_off, order_seq, mv, M, max_orders, max_lines, delta, status);
        if (rc != OR_OK) { free(delta); free(status); return rc; }
        int32_t best = -1;
        for (int32_t k = 0; k < M; ++k) {
            if (mv[4 * k + 3] != p || status[k] != 0 || delta[2 * k + 1] >= 0) continue;
            if (best < 0 || delta[2 * k + 1] < delta[2 * best + 1]) best = k;
        }
        if (best < 0) continue;
        applied[p] = best;
        const int32_t type = mv[4 * best], a = mv[4 * best + 1], b = mv[4 * best + 2];
        const int32_t t0 = plan_tour_off[p], t1 = plan_tour_off[p + 1];
        const int32_t s0 = tour_off[t0], s1 = tour_off[t1];
        if (type == 0) {
            int32_t ia = -1, ib = -1;
            for (int32_t q = s0; q < s1; ++q) {
                if (order_seq[q] == a) ia = q;
                if (order_seq[q] == b) ib = q;
            }
            order_seq[ia] = b;
            order_seq[ib] = a;
        } else if (type == 1) {
            int32_t ia = -1, ta = -1;
            for (int32_t t = t0; t < t1; ++t)
                for (int32_t q = tour_off[t]; q < tour_off[t + 1]; ++q)
                    if (order_seq[q] == a) { ia = q; ta = t; }
            const int32_t tb = t0 + b;
            if (tb > ta) {
                /* entries after a up to the end of tour tb move one place left */
                const int32_t end = tour_off[tb + 1];
                for (int32_t q = ia; q + 1 < end; ++q) order_seq[q] = order_seq[q + 1];
                order_seq[end - 1] = a;
                for (int32_t t = ta + 1; t <= tb; ++t) tour_off[t] -= 1;
            } else {
                /* entries from the end of tour tb up to a move one place right */
                const int32_t end = tour_off[tb + 1];
                for (int32_t q = ia; q > end; --q) order_seq[q] = order_seq[q - 1];
                order_seq[end] = a;
                for (int32_t t = tb + 1; t <= ta; ++t) tour_off[t] += 1;
            }
        } else if (type == 2) {
            int32_t *smap = slot_map + (int64_t)p * slot_map_stride;
            const int32_t tmp = smap[a];
            smap[a] = smap[b];
            smap[b] = tmp;
        } else {
            slot_map[(int64_t)p * slot_map_stride + a] = b;
        }
    }
    free(delta);
    free(status);
    return OR_OK;
}

/* ------------------------------------------------------- batch formation */

int or_batch_grow(const or_layout *g, int32_t n_orders, const int32_t *order_off, const int32_t *line_sku,
                  int32_t n_sku, const int32_t *slot_map, int32_t max_orders, int32_t max_lines,
                  int32_t *tour_off, int32_t *order_seq, int32_t *n_tours) {
    int rc = layout_check(g);
    if (rc != OR_OK) return rc;
    if (n_orders < 0 || max_orders < 0 || max_lines < 0) return OR_EINVAL;
    const int32_t n_loc = g->n_aisles * 2 * g->slots_per_side;
    const int32_t n_lines = n_orders > 0 ? order_off[n_orders] : 0;
    for (int32_t l = 0; l < n_lines; ++l) {
        const int32_t s = line_sku[l];
        if (s < 0 || s >= n_sku || slot_map[s] < 0 || slot_map[s] >= n_loc) return OR_ERANGE;
    }
    int32_t *locs = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_lines + 1));
    int64_t *alone = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_orders + 1));
    char *used = (char *)calloc((size_t)(n_orders + 1), 1);
    if (!locs || !alone || !used) { free(locs); free(alone); free(used); return OR_ENOMEM; }

    /* the length of each order's tour alone */
    for (int32_t o = 0; o < n_orders; ++o) {
        int32_t n = 0;
        for (int32_t l = order_off[o]; l < order_off[o + 1]; ++l) locs[n++] = slot_map[line_sku[l]];
        alone[o] = or_rr_tour(g, locs, n);
    }

    int32_t done = 0, tours = 0;
    tour_off[0] = 0;
    while (done < n_orders) {
        /* seed: the longest order alone */
        int32_t seed = -1;
        for (int32_t o = 0; o < n_orders; ++o)
            if (!used[o] && (seed < 0 || alone[o] > alone[seed])) seed = o;
        used[seed] = 1;
        order_seq[done++] = seed;
        int32_t n_tour = 0, lines = order_off[seed + 1] - order_off[seed], count = 1;
        for (int32_t l = order_off[seed]; l < order_off[seed + 1]; ++l) locs[n_tour++] = slot_map[line_sku[l]];
        int64_t cost = alone[seed];
        /* grow: the order that lengthens the tour least */
        while (max_orders == 0 || count < max_orders) {
            int32_t best = -1;
            int64_t best_cost = 0;
            for (int32_t o = 0; o < n_orders; ++o) {
                if (used[o]) continue;
                const int32_t ol = order_off[o + 1] - order_off[o];
                if (max_lines > 0 && lines + ol > max_lines) continue;
                int32_t n = n_tour;
                for (int32_t l = order_off[o]; l < order_off[o + 1]; ++l) locs[n++] = slot_map[line_sku[l]];
                const int64_t c = or_rr_tour(g, locs, n);
                if (best < 0 || c - cost < best_cost - cost) {
                    best = o;
                    best_cost = c;
                }
            }
            if (best < 0) break;
            used[best] = 1;
            order_seq[done++] = best;
            for (int32_t l = order_off[best]; l < order_off[best + 1]; ++l) locs[n_tour++] = slot_map[line_sku[l]];
            lines += order_off[best + 1] - order_off[best];
            ++count;
            cost = best_cost;
        }
        tour_off[++tours] = done;
    }
    *n_tours = tours;
    free(locs);
    free(alone);
    free(used);
    return OR_OK;
}

/* ------------------------------------------------------------- surrogate */

int or_features(const or_layout *g, const int32_t *locs, int32_t n, float *out) {
    int rc = layout_check(g);
    if (rc != OR_OK) return rc;
    for (int i = 0; i < 192; ++i) out[i] = 0.0f;
    const int32_t A = g->n_aisles, L = g->slots_per_side;
    int32_t *kmin = (int32_t *)malloc(sizeof(int32_t) * (size_t)A);
    int32_t *kmax = (int32_t *)malloc(sizeof(int32_t) * (size_t)A);
    if (!kmin || !kmax) { free(kmin); free(kmax); return OR_ENOMEM; }
    for (int32_t a = 0; a < A; ++a) { kmin[a] = -1; kmax[a] = -1; }
    for (int32_t i = 0; i < n; ++i) {
        const int32_t loc = locs[i];
        if (loc < 0 || loc >= A * 2 * L) { free(kmin); free(kmax); return OR_ERANGE; }
        const int32_t a = loc / (2 * L), k = loc % L;
        if (kmin[a] < 0 || k < kmin[a]) kmin[a] = k;
        if (k > kmax[a]) kmax[a] = k;
    }
    int32_t left = -1, right = -1, count = 0;
    for (int32_t a = 0; a < A; ++a) {
        if (kmax[a] < 0) continue;
        if (left < 0) left = a;
        right = a;
        ++count;
        out[(int64_t)kmax[a] * 64 / L] += 1.0f;
        out[64 + (int64_t)kmin[a] * 64 / L] += 1.0f;
        out[132 + (int64_t)a * 60 / A] += 1.0f;
    }
    const float inv_a = (float)(1.0 / (double)A);
    if (count > 0) {
        out[128] = (float)left * inv_a;
        out[129] = (float)right * inv_a;
    }
    out[130] = (float)count * inv_a;
    out[131] = (float)n * (1.0f / 64.0f);
    free(kmin);
    free(kmax);
    return OR_OK;
}

float or_bf16(float x) {
    uint32_t u;
    memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return x;          /* inf / nan: keep */
    const uint32_t lsb = (u >> 16) & 1u;
    u = (u + 0x7fffu + lsb) & 0xffff0000u;                   /* round to nearest even */
    float r;
    memcpy(&r, &u, 4);
    return r;
}

static double gelu(double x) { return 0.5 * x * (1.0 + erf(x / sqrt(2.0))); }
static double gelu_grad(double x) {
    return 0.5 * (1.0 + erf(x / sqrt(2.0))) + x * exp(-0.5 * x * x) / sqrt(2.0 * 3.14159265358979323846);
}

#define MLP_IN 192
#define MLP_H 256

/* forward for one row; z1, z2 pre-activations (double), h1, h2 bf16-rounded activations */
static double mlp_row(const float *w1, const float *b1, const float *w2, const float *b2, const float *w3,
                      const float *b3, const float *x, double *z1, double *h1, double *z2, double *h2) {
    for (int j = 0; j < MLP_H; ++j) {
        double s = b1[j];
        for (int i = 0; i < MLP_IN; ++i) s += (double)x[i] * (double)w1[i * MLP_H + j];
        z1[j] = s;
        h1[j] = (double)or_bf16((float)gelu(s));
    }
    for (int j = 0; j < MLP_H; ++j) {
        double s = b2[j];
        for (int i = 0; i < MLP_H; ++i) s += h1[i] * (double)w2[i * MLP_H + j];
        z2[j] = s;
        h2[j] = (double)or_bf16((float)gelu(s));
    }
    double y = b3[0];
    for (int i = 0; i < MLP_H; ++i) y += h2[i] * (double)w3[i];
    return y;
}

void or_mlp_forward(const float *w1, const float *b1, const float *w2, const float *b2, const float *w3,
                    const float *b3, const float *X, int32_t n, double *y) {
    double z1[MLP_H], h1[MLP_H], z2[MLP_H], h2[MLP_H];
    for (int32_t r = 0; r < n; ++r) y[r] = mlp_row(w1, b1, w2, b2, w3, b3, X + (int64_t)r * MLP_IN, z1, h1, z2, h2);
}

double or_mlp_backward(const float *w1, const float *b1, const float *w2, const float *b2, const float *w3,
                       const float *b3, const float *X, const double *t, int32_t n, double *g1, double *gb1,
                       double *g2, double *gb2, double *g3, double *gb3) {
    memset(g1, 0, sizeof(double) * MLP_IN * MLP_H);
    memset(gb1, 0, sizeof(double) * MLP_H);
    memset(g2, 0, sizeof(double) * MLP_H * MLP_H);
    memset(gb2, 0, sizeof(double) * MLP_H);
    memset(g3, 0, sizeof(double) * MLP_H);
    gb3[0] = 0.0;
    double z1[MLP_H], h1[MLP_H], z2[MLP_H], h2[MLP_H], d2[MLP_H], d1[MLP_H];
    double loss = 0.0;
    for (int32_t r = 0; r < n; ++r) {
        const float *x = X + (int64_t)r * MLP_IN;
        const double y = mlp_row(w1, b1, w2, b2, w3, b3, x, z1, h1, z2, h2);
        const double e = y - t[r];
        loss += 0.5 * e * e;
        const double dy = e / n;                  /* d loss / d y */
        gb3[0] += dy;
        for (int i = 0; i < MLP_H; ++i) {
            g3[i] += dy * h2[i];
            d2[i] = dy * (double)w3[i] * gelu_grad(z2[i]);   /* d loss / d z2 */
        }
        for (int j = 0; j < MLP_H; ++j) gb2[j] += d2[j];
        for (int i = 0; i < MLP_H; ++i) {
            double s = 0.0;
            for (int j = 0; j < MLP_H; ++j) {
                g2[i * MLP_H + j] += h1[i] * d2[j];
                s += (double)w2[i * MLP_H + j] * d2[j];
            }
            d1[i] = s * gelu_grad(z1[i]);                    /* d loss / d z1 */
        }
        for (int j = 0; j < MLP_H; ++j) gb1[j] += d1[j];
        for (int i = 0; i < MLP_IN; ++i)
            for (int j = 0; j < MLP_H; ++j) g1[i * MLP_H + j] += (double)x[i] * d1[j];
    }
    return loss / n;
}

/* One training step's every intermediate, row by row, with the rounding
 * points of the bf16-operand contract (bf16 weights and activations on the
 * tensor cores, fp32 accumulation; config 5 of the learned prescreen, the
 * paper's machine learning in the loop, Sec. 1 / Fig. 1): every operand of a
 * product is a bf16 value, so the forward's activations h1, h2 and the
 * backward's back-propagated pre-activation gradients d2 = dL/dz2 and
 * d1 = dL/dz1 are rounded to bf16 (through float, as the forward's
 * activations) before they are used; everything else is double.  The
 * gradients are the chain rule through that computation (each rounding
 * point passes the gradient through unchanged). */
double or_mlp_train_trace(const float *w1, const float *b1, const float *w2, const float *b2, const float *w3,
                          const float *b3, const float *X, const double *t, int32_t n, double *z1, double *h1,
                          double *z2, double *h2, double *y, double *dy, double *d2pre, double *d2, double *s1,
                          double *d1pre, double *d1, double *g1, double *gb1, double *g2, double *gb2, double *g3,
                          double *gb3) {
    memset(g1, 0, sizeof(double) * MLP_IN * MLP_H);
    memset(gb1, 0, sizeof(double) * MLP_H);
    memset(g2, 0, sizeof(double) * MLP_H * MLP_H);
    memset(gb2, 0, sizeof(double) * MLP_H);
    memset(g3, 0, sizeof(double) * MLP_H);
    gb3[0] = 0.0;
    double loss = 0.0;
    for (int32_t r = 0; r < n; ++r) {
        const int64_t o = (int64_t)r * MLP_H;
        const float *x = X + (int64_t)r * MLP_IN;
        y[r] = mlp_row(w1, b1, w2, b2, w3, b3, x, z1 + o, h1 + o, z2 + o, h2 + o);
        const double e = y[r] - t[r];
        loss += 0.5 * e * e;
        dy[r] = e / n;
        gb3[0] += dy[r];
        for (int i = 0; i < MLP_H; ++i) {
            g3[i] += dy[r] * h2[o + i];
            d2pre[o + i] = dy[r] * (double)w3[i] * gelu_grad(z2[o + i]);
            d2[o + i] = (double)or_bf16((float)d2pre[o + i]);
        }
        for (int j = 0; j < MLP_H; ++j) gb2[j] += d2[o + j];
        for (int i = 0; i < MLP_H; ++i) {
            double acc = 0.0;
            for (int j = 0; j < MLP_H; ++j) {
                g2[i * MLP_H + j] += h1[o + i] * d2[o + j];
                acc += (double)w2[i * MLP_H + j] * d2[o + j];
            }
            s1[o + i] = acc;
            d1pre[o + i] = acc * gelu_grad(z1[o + i]);
            d1[o + i] = (double)or_bf16((float)d1pre[o + i]);
        }
        for (int j = 0; j < MLP_H; ++j) gb1[j] += d1[o + j];
        for (int i = 0; i < MLP_IN; ++i)
            for (int j = 0; j < MLP_H; ++j) g1[i * MLP_H + j] += (double)x[i] * d1[o + j];
    }
    return loss / n;
}

void or_adam(double *p, double *m, double *v, const double *g, int64_t n, double lr, double b1, double b2,
             double eps, int32_t step) {
    const double c1 = 1.0 - pow(b1, step), c2 = 1.0 - pow(b2, step);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        p[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
}

/* ------------------------------------------------------------ K-means slotting
 * Subproblem 3 (Sec. 5): product placement by picking frequency, with an
 * unsupervised K-means classification (MacQueen 1967) deciding which products
 * are stored together; the reading's steps, in order, are in the header. */

static int64_t floor_div64(int64_t a, int64_t b) { /* b > 0 */
    int64_t q = a / b;
    if ((a % b) != 0 && a < 0) --q;
    return q;
}

/* floor(sqrt(v)) exactly: a floating-point estimate corrected by integer
 * comparisons */
static int64_t isqrt64(int64_t v) {
    int64_t r = (int64_t)sqrt((double)v);
    while (r > 0 && r * r > v) --r;
    while ((r + 1) * (r + 1) <= v) ++r;
    return r;
}

static int32_t bitlen32(int32_t v) {
    int32_t b = 0;
    while (v > 0) { ++b; v >>= 1; }
    return b;
}

static int64_t sqdist(const int32_t *x, const int32_t *c) {
    int64_t d = 0;
    for (int j = 0; j < OR_KM_DIM; ++j) {
        const int64_t e = (int64_t)x[j] - (int64_t)c[j];
        d += e * e;
    }
    return d;
}

static int32_t nearest(const int32_t *x, const int32_t *cent, int32_t k) {
    int32_t best = 0;
    int64_t bd = sqdist(x, cent);
    for (int32_t c = 1; c < k; ++c) {
        const int64_t d = sqdist(x, cent + (int64_t)c * OR_KM_DIM);
        if (d < bd) { bd = d; best = c; }   /* ties: the lowest cluster */
    }
    return best;
}

typedef struct {
    int64_t cluster_rank, freq;
    int32_t sku;
} km_key_t;

static int cmp_km_key(const void *p, const void *q) {
    const km_key_t *a = (const km_key_t *)p, *b = (const km_key_t *)q;
    if (a->cluster_rank != b->cluster_rank) return a->cluster_rank < b->cluster_rank ? -1 : 1;
    if (a->freq != b->freq) return a->freq > b->freq ? -1 : 1;   /* more picks first */
    return a->sku < b->sku ? -1 : (a->sku > b->sku);
}

typedef struct {
    int64_t weight;
    int32_t cluster;
} km_cluster_t;

static int cmp_km_cluster(const void *p, const void *q) {
    const km_cluster_t *a = (const km_cluster_t *)p, *b = (const km_cluster_t *)q;
    if (a->weight != b->weight) return a->weight > b->weight ? -1 : 1;   /* heavier first */
    return a->cluster < b->cluster ? -1 : (a->cluster > b->cluster);
}

int or_kmeans_features(int32_t n_orders, const int32_t *order_off, const int32_t *line_sku, int32_t n_sku,
                       const int8_t *signs, int32_t freq_weight, int32_t *x, int32_t *freq) {
    if (n_orders < 0 || n_sku < 1 || !order_off || !signs || !x || !freq) return OR_EINVAL;
    int64_t *co = (int64_t *)calloc((size_t)n_sku * OR_KM_DIM, sizeof(int64_t));
    if (!co) return OR_ENOMEM;
    memset(freq, 0, sizeof(int32_t) * (size_t)n_sku);
    int rc = OR_OK;
    for (int32_t o = 0; o < n_orders && rc == OR_OK; ++o) {
        const int32_t lb = order_off[o], le = order_off[o + 1];
        if (lb < 0 || le < lb) { rc = OR_EINVAL; break; }
        for (int32_t l = lb; l < le; ++l) {
            const int32_t s = line_sku[l];
            if (s < 0 || s >= n_sku) { rc = OR_ERANGE; break; }
            ++freq[s];
            /* co-occurrence row of s, projected: every other line of the order */
            for (int32_t m = lb; m < le; ++m) {
                if (m == l) continue;
                const int32_t t = line_sku[m];
                if (t < 0 || t >= n_sku) { rc = OR_ERANGE; break; }
                for (int j = 0; j < OR_KM_SKETCH; ++j) co[(int64_t)s * OR_KM_DIM + j] += signs[(int64_t)t * OR_KM_DIM + j];
            }
        }
    }
    for (int32_t s = 0; s < n_sku && rc == OR_OK; ++s) {
        const int64_t *c = co + (int64_t)s * OR_KM_DIM;
        int64_t nn = 0;
        for (int j = 0; j < OR_KM_SKETCH; ++j) nn += c[j] * c[j];
        const int64_t n = isqrt64(nn);
        int32_t *xs = x + (int64_t)s * OR_KM_DIM;
        for (int j = 0; j < OR_KM_SKETCH; ++j) xs[j] = n > 0 ? (int32_t)(c[j] * OR_KM_SCALE / n) : 0;
        xs[OR_KM_SKETCH] = freq_weight * bitlen32(freq[s]);
    }
    free(co);
    return rc;
}

int or_kmeans_lloyd(const int32_t *x, int32_t n, int32_t k, int32_t iters, int32_t *centroids, int32_t *assign) {
    if (n < 1 || k < 1 || iters < 0 || !x || !centroids || !assign) return OR_EINVAL;
    int64_t *sum = (int64_t *)malloc(sizeof(int64_t) * (size_t)k * OR_KM_DIM);
    int64_t *cnt = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
    if (!sum || !cnt) { free(sum); free(cnt); return OR_ENOMEM; }
    for (int32_t it = 0; it < iters; ++it) {
        /* assignment: the nearest centroid */
        memset(sum, 0, sizeof(int64_t) * (size_t)k * OR_KM_DIM);
        memset(cnt, 0, sizeof(int64_t) * (size_t)k);
        for (int32_t s = 0; s < n; ++s) {
            const int32_t c = nearest(x + (int64_t)s * OR_KM_DIM, centroids, k);
            ++cnt[c];
            for (int j = 0; j < OR_KM_DIM; ++j) sum[(int64_t)c * OR_KM_DIM + j] += x[(int64_t)s * OR_KM_DIM + j];
        }
        /* update: the members' mean, rounded to the nearest integer (halves up) */
        for (int32_t c = 0; c < k; ++c) {
            if (cnt[c] == 0) continue;
            for (int j = 0; j < OR_KM_DIM; ++j)
                centroids[(int64_t)c * OR_KM_DIM + j] =
                    (int32_t)floor_div64(2 * sum[(int64_t)c * OR_KM_DIM + j] + cnt[c], 2 * cnt[c]);
        }
    }
    for (int32_t s = 0; s < n; ++s) assign[s] = nearest(x + (int64_t)s * OR_KM_DIM, centroids, k);
    free(sum);
    free(cnt);
    return OR_OK;
}

int or_kmeans_pp_init(const int32_t *x, int32_t n, int32_t k, const uint64_t *u, int32_t *init) {
    if (n < 1 || k < 1 || k > n || !x || !u || !init) return OR_EINVAL;
    int64_t *d = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (!d) return OR_ENOMEM;
    init[0] = (int32_t)(u[0] % (uint64_t)n);
    for (int32_t s = 0; s < n; ++s) d[s] = sqdist(x + (int64_t)s * OR_KM_DIM, x + (int64_t)init[0] * OR_KM_DIM);
    for (int32_t c = 1; c < k; ++c) {
        int64_t total = 0;
        for (int32_t s = 0; s < n; ++s) total += d[s];
        int32_t pick;
        if (total == 0) {
            pick = (int32_t)(u[c] % (uint64_t)n);
        } else {
            /* the SKU whose share of the running sum of D^2 covers the draw */
            const int64_t target = (int64_t)(u[c] % (uint64_t)total);
            int64_t run = 0;
            pick = n - 1;
            for (int32_t s = 0; s < n; ++s) {
                run += d[s];
                if (run > target) { pick = s; break; }
            }
        }
        init[c] = pick;
        for (int32_t s = 0; s < n; ++s) {
            const int64_t e = sqdist(x + (int64_t)s * OR_KM_DIM, x + (int64_t)pick * OR_KM_DIM);
            if (e < d[s]) d[s] = e;
        }
    }
    free(d);
    return OR_OK;
}

int or_kmeans_slotting(const or_layout *g, int32_t n_orders, const int32_t *order_off, const int32_t *line_sku,
                       int32_t n_sku, const int8_t *signs, int32_t freq_weight, int32_t k, const int32_t *init,
                       const uint64_t *u, int32_t iters, int32_t *x_out, int32_t *init_out, int32_t *centroids,
                       int32_t *assign, int32_t *slot_map) {
    int rc = layout_check(g);
    if (rc != OR_OK) return rc;
    if (k < 1 || k > n_sku || iters < 0 || freq_weight < 0 || freq_weight > OR_KM_MAX_FREQ_WEIGHT ||
        (!init && !u) || !centroids || !assign || !slot_map)
        return OR_EINVAL;
    const int64_t n_loc = (int64_t)g->n_aisles * 2 * g->slots_per_side;
    if (n_sku > n_loc) return OR_ERANGE;
    int32_t *x = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_sku * OR_KM_DIM);
    int32_t *freq = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_sku);
    km_cluster_t *cl = (km_cluster_t *)malloc(sizeof(km_cluster_t) * (size_t)k);
    int64_t *cl_rank = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
    km_key_t *keys = (km_key_t *)malloc(sizeof(km_key_t) * (size_t)n_sku);
    int32_t *seed = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
    if (!x || !freq || !cl || !cl_rank || !keys || !seed) { rc = OR_ENOMEM; goto done; }
    /* 1-2: features */
    rc = or_kmeans_features(n_orders, order_off, line_sku, n_sku, signs, freq_weight, x, freq);
    if (rc != OR_OK) goto done;
    /* 3: initial centroids: the given SKUs, else K-means++ seeding */
    if (init) {
        memcpy(seed, init, sizeof(int32_t) * (size_t)k);
    } else {
        rc = or_kmeans_pp_init(x, n_sku, k, u, seed);
        if (rc != OR_OK) goto done;
    }
    for (int32_t c = 0; c < k; ++c) {
        if (seed[c] < 0 || seed[c] >= n_sku) { rc = OR_ERANGE; goto done; }
        memcpy(centroids + (int64_t)c * OR_KM_DIM, x + (int64_t)seed[c] * OR_KM_DIM, sizeof(int32_t) * OR_KM_DIM);
    }
    if (init_out) memcpy(init_out, seed, sizeof(int32_t) * (size_t)k);
    /* 4: Lloyd rounds */
    rc = or_kmeans_lloyd(x, n_sku, k, iters, centroids, assign);
    if (rc != OR_OK) goto done;
    /* 5: cluster weight = picks of its members (the final assignment) */
    for (int32_t c = 0; c < k; ++c) { cl[c].weight = 0; cl[c].cluster = c; }
    for (int32_t s = 0; s < n_sku; ++s) cl[assign[s]].weight += freq[s];
    /* 6: zones: clusters by weight (heavier first, ties lowest id); SKUs by
     * (their cluster's rank, more picks first, lower id) */
    qsort(cl, (size_t)k, sizeof(km_cluster_t), cmp_km_cluster);
    for (int32_t r = 0; r < k; ++r) cl_rank[cl[r].cluster] = r;
    for (int32_t s = 0; s < n_sku; ++s) {
        keys[s].cluster_rank = cl_rank[assign[s]];
        keys[s].freq = freq[s];
        keys[s].sku = s;
    }
    qsort(keys, (size_t)n_sku, sizeof(km_key_t), cmp_km_key);
    /* 7: the r-th SKU takes the r-th location in aisle-major order: aisle,
     * then depth from the front, then side */
    for (int32_t r = 0; r < n_sku; ++r) {
        const int32_t L = g->slots_per_side;
        const int32_t a = r / (2 * L), q = r % (2 * L), depth = q / 2, side = q % 2;
        slot_map[keys[r].sku] = (a * 2 + side) * L + depth;
    }
    if (x_out) memcpy(x_out, x, sizeof(int32_t) * (size_t)n_sku * OR_KM_DIM);
done:
    free(x); free(freq); free(cl); free(cl_rank); free(keys); free(seed);
    return rc;
}
