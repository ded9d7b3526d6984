/*
 * Seeded synthetic-input generator for the warehouse plan evaluator.
 *
 * This file produces INPUTS only: order books, SKU-to-location slottings,
 * candidate plans (partitions of the orders into picker tours) and
 * neighbourhood moves.  It holds none of the tour-cost arithmetic; both the
 * CPU oracle and the CUDA path consume the arrays it writes.
 *
 * Workload shapes follow the paper's scale statement (Sec. 1: ~10,000 items a
 * day over ~4,000 orders and up to 200,000 locations) and the order-picking
 * problem statement of Sec. 5 (order history o, product position x, picking
 * list).  The distributions below are the readings recorded in the design
 * notes: truncated-geometric order sizes, Zipf SKU popularity, ABC slotting
 * with random transpositions, random partitions into capacity-capped tours.
 *
 * Random numbers: SplitMix64 (Steele, Lea & Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), one counter-seeded stream per
 * (seed, tag, index).  Integer ranges use the multiply-shift map
 * (u32 * n) >> 32.  Plain C99, no platform intrinsics.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define GEN_OK 0
#define GEN_EINVAL -1
#define GEN_ENOMEM -3

/* stream tags */
#define TAG_ORDER_SIZE 1u
#define TAG_ORDER_SKU 2u
#define TAG_SLOT 3u
#define TAG_SWAP 4u
#define TAG_PLAN 5u
#define TAG_MOVE 6u
#define TAG_INST 7u
#define TAG_CATEGORY 8u
#define TAG_SIGN 9u
#define TAG_RELOC 10u

typedef struct { uint64_t s; } rng_t;

static uint64_t sm64_next(rng_t *r) {
    uint64_t z = (r->s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* independent stream for (seed, tag, idx): the seed words are themselves
 * passed through the SplitMix64 finaliser so that neighbouring indices give
 * unrelated streams */
static rng_t stream(uint64_t seed, uint32_t tag, uint64_t idx) {
    rng_t r;
    r.s = seed;
    uint64_t a = sm64_next(&r);
    r.s = a ^ ((uint64_t)tag << 40) ^ 0x5851F42D4C957F2Dull;
    uint64_t b = sm64_next(&r);
    r.s = b ^ idx;
    (void)sm64_next(&r);
    return r;
}

static uint32_t u32(rng_t *r) { return (uint32_t)(sm64_next(r) >> 32); }
/* uniform integer in [0, n) */
static int32_t below(rng_t *r, int32_t n) { return (int32_t)(((uint64_t)u32(r) * (uint64_t)n) >> 32); }
/* uniform double in [0, 1) */
static double unit(rng_t *r) { return (double)(sm64_next(r) >> 11) * (1.0 / 9007199254740992.0); }

/* first index i with cdf[i] > u (cdf strictly increasing to 1) */
static int32_t cdf_search(const double *cdf, int32_t n, double u) {
    int32_t lo = 0, hi = n - 1;
    while (lo < hi) {
        int32_t mid = lo + (hi - lo) / 2;
        if (cdf[mid] > u) hi = mid; else lo = mid + 1;
    }
    return lo;
}

/* ------------------------------------------------------------------ orders */

/* Orders with sizes drawn from a truncated geometric law on 1..max_lines,
 * P(k) proportional to (1-p)^(k-1), and distinct SKUs per order drawn either
 * uniformly (zipf_s <= 0) or by Zipf popularity P(rank i) ~ i^-s (SKU id =
 * rank - 1, so SKU 0 is the most popular).  Writes order_off[n_orders+1] and
 * line_sku[..]; line_cap must be >= n_orders*max_lines.  Returns the number of
 * lines, or a negative error. */
int64_t gen_orders(uint64_t seed, int32_t n_orders, int32_t n_sku, int32_t max_lines,
                   double p_geom, double zipf_s, int32_t *order_off, int32_t *line_sku,
                   int64_t line_cap) {
    if (n_orders < 0 || n_sku <= 0 || max_lines <= 0 || max_lines > n_sku ||
        !(p_geom > 0.0 && p_geom <= 1.0))
        return GEN_EINVAL;
    if ((int64_t)n_orders * max_lines > line_cap) return GEN_EINVAL;
    double *size_cdf = (double *)malloc(sizeof(double) * (size_t)max_lines);
    double *sku_cdf = NULL;
    if (!size_cdf) return GEN_ENOMEM;
    double acc = 0.0, w = 1.0;
    for (int32_t k = 0; k < max_lines; ++k) { acc += w; size_cdf[k] = acc; w *= (1.0 - p_geom); }
    for (int32_t k = 0; k < max_lines; ++k) size_cdf[k] /= acc;
    size_cdf[max_lines - 1] = 2.0; /* guard against rounding */
    if (zipf_s > 0.0) {
        sku_cdf = (double *)malloc(sizeof(double) * (size_t)n_sku);
        if (!sku_cdf) { free(size_cdf); return GEN_ENOMEM; }
        double z = 0.0;
        for (int32_t i = 0; i < n_sku; ++i) { z += pow((double)(i + 1), -zipf_s); sku_cdf[i] = z; }
        for (int32_t i = 0; i < n_sku; ++i) sku_cdf[i] /= z;
        sku_cdf[n_sku - 1] = 2.0;
    }
    int64_t pos = 0;
    order_off[0] = 0;
    for (int32_t o = 0; o < n_orders; ++o) {
        rng_t rs = stream(seed, TAG_ORDER_SIZE, (uint64_t)o);
        int32_t k = cdf_search(size_cdf, max_lines, unit(&rs)) + 1;
        rng_t rk = stream(seed, TAG_ORDER_SKU, (uint64_t)o);
        for (int32_t j = 0; j < k; ++j) {
            int32_t sku;
            for (;;) { /* distinct SKUs within one order: redraw on repeat */
                sku = sku_cdf ? cdf_search(sku_cdf, n_sku, unit(&rk)) : below(&rk, n_sku);
                int dup = 0;
                for (int64_t q = pos - j; q < pos; ++q) if (line_sku[q] == sku) { dup = 1; break; }
                if (!dup) break;
            }
            line_sku[pos++] = sku;
        }
        order_off[o + 1] = (int32_t)pos;
    }
    free(size_cdf);
    free(sku_cdf);
    return pos;
}

/* Orders with a category structure (the paper's retail case study clusters
 * "different categories"): SKU s belongs to category s mod n_cat, so every
 * category holds SKUs of every popularity.  Each order draws its category
 * uniformly, a size as gen_orders, and each line: with probability p_in the
 * i-th SKU of the order's category with Zipf popularity P(i) ~ (i+1)^-s over
 * the first floor(n_sku / n_cat) members (SKU id = category + i * n_cat),
 * otherwise a SKU of the whole catalogue by Zipf popularity (SKU id = rank).
 * SKUs are distinct within an order (redraw on repeat).  Same outputs and
 * return value as gen_orders. */
int64_t gen_orders_cat(uint64_t seed, int32_t n_orders, int32_t n_sku, int32_t max_lines, double p_geom,
                       double zipf_s, int32_t n_cat, double p_in, int32_t *order_off, int32_t *line_sku,
                       int64_t line_cap) {
    if (n_orders < 0 || n_sku <= 0 || max_lines <= 0 || n_cat <= 0 || n_cat > n_sku || !(zipf_s > 0.0) ||
        !(p_geom > 0.0 && p_geom <= 1.0) || !(p_in >= 0.0 && p_in <= 1.0))
        return GEN_EINVAL;
    const int32_t per_cat = n_sku / n_cat;
    if (max_lines > per_cat || (int64_t)n_orders * max_lines > line_cap) return GEN_EINVAL;
    double *size_cdf = (double *)malloc(sizeof(double) * (size_t)max_lines);
    double *sku_cdf = (double *)malloc(sizeof(double) * (size_t)n_sku);
    double *cat_cdf = (double *)malloc(sizeof(double) * (size_t)per_cat);
    if (!size_cdf || !sku_cdf || !cat_cdf) {
        free(size_cdf); free(sku_cdf); free(cat_cdf);
        return GEN_ENOMEM;
    }
    double acc = 0.0, w = 1.0;
    for (int32_t k = 0; k < max_lines; ++k) { acc += w; size_cdf[k] = acc; w *= (1.0 - p_geom); }
    for (int32_t k = 0; k < max_lines; ++k) size_cdf[k] /= acc;
    size_cdf[max_lines - 1] = 2.0;
    double z = 0.0;
    for (int32_t i = 0; i < n_sku; ++i) { z += pow((double)(i + 1), -zipf_s); sku_cdf[i] = z; }
    for (int32_t i = 0; i < n_sku; ++i) sku_cdf[i] /= z;
    sku_cdf[n_sku - 1] = 2.0;
    z = 0.0;
    for (int32_t i = 0; i < per_cat; ++i) { z += pow((double)(i + 1), -zipf_s); cat_cdf[i] = z; }
    for (int32_t i = 0; i < per_cat; ++i) cat_cdf[i] /= z;
    cat_cdf[per_cat - 1] = 2.0;
    int64_t pos = 0;
    order_off[0] = 0;
    for (int32_t o = 0; o < n_orders; ++o) {
        rng_t rs = stream(seed, TAG_ORDER_SIZE, (uint64_t)o);
        int32_t k = cdf_search(size_cdf, max_lines, unit(&rs)) + 1;
        rng_t rc = stream(seed, TAG_CATEGORY, (uint64_t)o);
        const int32_t cat = below(&rc, n_cat);
        rng_t rk = stream(seed, TAG_ORDER_SKU, (uint64_t)o);
        for (int32_t j = 0; j < k; ++j) {
            int32_t sku;
            for (;;) {
                if (unit(&rk) < p_in) sku = cat + cdf_search(cat_cdf, per_cat, unit(&rk)) * n_cat;
                else sku = cdf_search(sku_cdf, n_sku, unit(&rk));
                int dup = 0;
                for (int64_t q = pos - j; q < pos; ++q) if (line_sku[q] == sku) { dup = 1; break; }
                if (!dup) break;
            }
            line_sku[pos++] = sku;
        }
        order_off[o + 1] = (int32_t)pos;
    }
    free(size_cdf);
    free(sku_cdf);
    free(cat_cdf);
    return pos;
}

/* n values in {-1, +1}, each from one bit of stream (seed, TAG_SIGN, i / 64) --
 * the random sign matrix of a sketch, drawn by the caller and passed in. */
int gen_signs(uint64_t seed, int64_t n, int8_t *out) {
    if (n < 0) return GEN_EINVAL;
    for (int64_t i = 0; i < n; i += 64) {
        rng_t r = stream(seed, TAG_SIGN, (uint64_t)(i / 64));
        const uint64_t bits = sm64_next(&r);
        for (int64_t b = 0; b < 64 && i + b < n; ++b) out[i + b] = (int8_t)(((bits >> b) & 1u) ? 1 : -1);
    }
    return GEN_OK;
}

/* ---------------------------------------------------------------- slotting */

/* Random injective slotting: SKU s goes to the s-th entry of a uniformly
 * random permutation of the n_loc location ids. */
int gen_slot_random(uint64_t seed, int32_t n_sku, int32_t n_loc, int32_t *slot_map) {
    if (n_sku <= 0 || n_loc < n_sku) return GEN_EINVAL;
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_loc);
    if (!perm) return GEN_ENOMEM;
    for (int32_t i = 0; i < n_loc; ++i) perm[i] = i;
    rng_t r = stream(seed, TAG_SLOT, 0);
    for (int32_t i = n_loc - 1; i > 0; --i) {
        int32_t j = below(&r, i + 1);
        int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
    memcpy(slot_map, perm, sizeof(int32_t) * (size_t)n_sku);
    free(perm);
    return GEN_OK;
}

typedef struct { int64_t rank_key; int32_t loc; } loc_rank_t;

static int cmp_loc_rank(const void *a, const void *b) {
    const loc_rank_t *x = (const loc_rank_t *)a, *y = (const loc_rank_t *)b;
    if (x->rank_key != y->rank_key) return x->rank_key < y->rank_key ? -1 : 1;
    return x->loc < y->loc ? -1 : (x->loc > y->loc);
}

/* ABC slotting: locations are ranked by their walking distance from the depot
 * along the front cross-aisle (aisle_index * aisle_pitch + slot depth, with the
 * slot depth W/2 + k*S), ties by location id; the SKU of popularity rank i
 * (SKU id i) takes the location of rank i.  Then floor(swap_frac*n_sku/2)
 * random transpositions of two SKUs' slots.  Location id encoding:
 * loc = (aisle*2 + side)*L + k. */
int gen_slot_abc(uint64_t seed, int32_t n_aisles, int32_t slots_per_side, int32_t aisle_pitch,
                 int32_t slot_pitch, int32_t cross_aisle_width, int32_t n_sku, double swap_frac,
                 int32_t *slot_map) {
    int64_t n_loc = (int64_t)n_aisles * 2 * slots_per_side;
    if (n_sku <= 0 || n_loc < n_sku || n_loc > 0x7fffffff) return GEN_EINVAL;
    loc_rank_t *lr = (loc_rank_t *)malloc(sizeof(loc_rank_t) * (size_t)n_loc);
    if (!lr) return GEN_ENOMEM;
    for (int64_t loc = 0; loc < n_loc; ++loc) {
        int64_t a = loc / (2 * (int64_t)slots_per_side);
        int64_t k = loc % slots_per_side;
        lr[loc].rank_key = a * aisle_pitch + cross_aisle_width / 2 + k * slot_pitch;
        lr[loc].loc = (int32_t)loc;
    }
    qsort(lr, (size_t)n_loc, sizeof(loc_rank_t), cmp_loc_rank);
    for (int32_t s = 0; s < n_sku; ++s) slot_map[s] = lr[s].loc;
    free(lr);
    int64_t n_swaps = (int64_t)floor(swap_frac * (double)n_sku / 2.0);
    rng_t r = stream(seed, TAG_SWAP, 0);
    for (int64_t q = 0; q < n_swaps; ++q) {
        int32_t i = below(&r, n_sku), j = below(&r, n_sku);
        int32_t t = slot_map[i]; slot_map[i] = slot_map[j]; slot_map[j] = t;
    }
    return GEN_OK;
}

/* ------------------------------------------------------------------- plans */

static void shuffle_orders(rng_t *r, int32_t *seq, int32_t n) {
    for (int32_t i = 0; i < n; ++i) seq[i] = i;
    for (int32_t i = n - 1; i > 0; --i) {
        int32_t j = below(r, i + 1);
        int32_t t = seq[i]; seq[i] = seq[j]; seq[j] = t;
    }
}

/* Candidate plans.  Each plan is a uniformly random order sequence cut into
 * tours.  mode 0: chunks of U{1..max_orders} orders.  mode 1: greedy fill,
 * closing a tour before it would exceed max_orders orders or max_lines lines
 * (max_lines <= 0: no line cap).  Outputs are global CSR arrays over all plans:
 * plan_tour_off[n_plans+1] indexes tours, tour_off[n_tours+1] indexes
 * order_seq[n_plans*n_orders].  Plan p draws from stream (seed, PLAN, plan_base+p).
 * tour_cap bounds the number of tours.  Returns n_tours or a negative error. */
int64_t gen_plans(uint64_t seed, int32_t mode, const int32_t *order_off, int32_t n_orders,
                  int32_t n_plans, int64_t plan_base, int32_t max_orders, int32_t max_lines,
                  int32_t *plan_tour_off, int32_t *tour_off, int32_t *order_seq,
                  int64_t tour_cap) {
    if (n_orders < 0 || n_plans < 0 || max_orders <= 0) return GEN_EINVAL;
    if ((int64_t)n_plans * n_orders > 0x7fffffff) return GEN_EINVAL;
    int64_t nt = 0;
    plan_tour_off[0] = 0;
    tour_off[0] = 0;
    for (int32_t p = 0; p < n_plans; ++p) {
        rng_t r = stream(seed, TAG_PLAN, (uint64_t)(plan_base + p));
        int32_t *seq = order_seq + (int64_t)p * n_orders;
        shuffle_orders(&r, seq, n_orders);
        int64_t base = (int64_t)p * n_orders;
        int32_t i = 0;
        while (i < n_orders) {
            int32_t take;
            if (mode == 0) {
                take = below(&r, max_orders) + 1;
                if (take > n_orders - i) take = n_orders - i;
            } else {
                int32_t lines = 0;
                take = 0;
                while (i + take < n_orders && take < max_orders) {
                    int32_t o = seq[i + take];
                    int32_t l = order_off[o + 1] - order_off[o];
                    if (max_lines > 0 && take > 0 && lines + l > max_lines) break;
                    lines += l;
                    ++take;
                }
            }
            if (nt >= tour_cap) return GEN_EINVAL;
            i += take;
            tour_off[++nt] = (int32_t)(base + i);
        }
        plan_tour_off[p + 1] = (int32_t)nt;
    }
    return nt;
}

/* ------------------------------------------------------------------- moves */

/* Neighbourhood moves for plan-level local search, four int32 per move:
 * {type, a, b, 0}.  type 0 = swap orders a and b between their tours,
 * type 1 = relocate order a into tour b (tour index local to the plan),
 * type 2 = swap the slots of SKUs a and b.  The type is uniform over the
 * three kinds; order ids are uniform over the orders; the target tour is
 * uniform over the plan's tours; SKU a is uniform over the SKUs that occur in
 * the order book (sku_pool), SKU b uniform over all SKUs.  Move (p, k) draws
 * from stream (seed, MOVE, (step << 32) ^ (p << 8) ^ k) so that any move can be
 * regenerated on its own. */
int gen_moves(uint64_t seed, int64_t step, int32_t n_plans, int32_t moves_per_plan,
              int32_t n_orders, const int32_t *plan_n_tours, const int32_t *sku_pool,
              int32_t pool_n, int32_t n_sku, int32_t *moves) {
    if (n_orders <= 1 || moves_per_plan <= 0 || moves_per_plan > 256 || n_sku <= 1 || pool_n <= 0)
        return GEN_EINVAL;
    for (int32_t p = 0; p < n_plans; ++p) {
        for (int32_t k = 0; k < moves_per_plan; ++k) {
            rng_t r = stream(seed, TAG_MOVE,
                             ((uint64_t)step << 32) ^ ((uint64_t)p << 8) ^ (uint64_t)k);
            int32_t *m = moves + ((int64_t)p * moves_per_plan + k) * 4;
            int32_t type = below(&r, 3);
            m[0] = type;
            m[3] = 0;
            if (type == 0) {
                m[1] = below(&r, n_orders);
                m[2] = below(&r, n_orders);
            } else if (type == 1) {
                m[1] = below(&r, n_orders);
                m[2] = below(&r, plan_n_tours[p] > 0 ? plan_n_tours[p] : 1);
            } else {
                m[1] = sku_pool[below(&r, pool_n)];
                m[2] = below(&r, n_sku);
            }
        }
    }
    return GEN_OK;
}

/* Relocation moves {3, sku, location, plan}: the SKU drawn from sku_pool
 * (SKUs that appear in orders), the target location uniform over the n_loc
 * locations (occupied targets are the evaluator's to reject); plan = the
 * plan index. */
int gen_relocations(uint64_t seed, int64_t step, int32_t n_plans, int32_t moves_per_plan,
                    const int32_t *sku_pool, int32_t pool_n, int32_t n_loc, int32_t *moves) {
    if (moves_per_plan <= 0 || moves_per_plan > 256 || pool_n <= 0 || n_loc <= 0) return GEN_EINVAL;
    for (int32_t p = 0; p < n_plans; ++p) {
        for (int32_t k = 0; k < moves_per_plan; ++k) {
            rng_t r = stream(seed, TAG_RELOC, ((uint64_t)step << 32) ^ ((uint64_t)p << 8) ^ (uint64_t)k);
            int32_t *m = moves + ((int64_t)p * moves_per_plan + k) * 4;
            m[0] = 3;
            m[1] = sku_pool[below(&r, pool_n)];
            m[2] = below(&r, n_loc);
            m[3] = p;
        }
    }
    return GEN_OK;
}

/* Uniform integer in [lo, hi] for instance-level parameters (batched workloads). */
int32_t gen_instance_param(uint64_t seed, int64_t inst, int32_t which, int32_t lo, int32_t hi) {
    rng_t r = stream(seed, TAG_INST, ((uint64_t)inst << 4) ^ (uint64_t)which);
    return lo + below(&r, hi - lo + 1);
}

/* raw SplitMix64 draw of stream (seed, tag, idx), word n; exposed so that the
 * stream derivation itself can be checked */
uint64_t gen_stream_word(uint64_t seed, uint32_t tag, uint64_t idx, int32_t n) {
    rng_t r = stream(seed, tag, idx);
    uint64_t v = 0;
    for (int32_t i = 0; i <= n; ++i) v = sm64_next(&r);
    return v;
}
