/*
 * CPU ORACLE for the warehouse plan evaluator -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded C evaluator of order-picking tour lengths,
 * written to be checked against the paper by eye.  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may load it; the product
 * path (the CUDA library) never links, calls or includes anything here, and
 * this file includes nothing of the product path.
 *
 * What it follows:
 *   Sec. 5, Eq. (2): subproblem 2 minimises the picking route sum d_i; the
 *     distance between two picking positions is a shortest path (the paper
 *     names Dijkstra) and the route is the best permutation of the picking
 *     sequence.  The oracle computes, per tour,
 *       - the S-shape route length (a fixed routing rule, simulated walk),
 *       - the optimal route length by the Ratliff-Rosenthal aisle-by-aisle
 *         dynamic programme (Ratliff & Rosenthal, Oper. Res. 31(3), 1983),
 *       - for small tours, the optimum by Held-Karp and by enumerating
 *         permutations of the picking sequence (the paper's own wording).
 *   Sec. 5: a plan = product positions x (slot map) + picking lists (which
 *     orders are picked together); its cost is the sum of its tours' lengths.
 *   Sec. 5, subroutine 4 / picking list: a move changes one plan; its delta
 *     is the plan cost after the move minus before (plain re-evaluation).
 *
 * Geometry (the paper gives none; reading used throughout): aisle a has its
 * centreline at x_a = a*P; slot k (either side) is at depth y_k = W/2 + k*S;
 * the front cross-aisle centre is depth 0, the back one Y = W + (L-1)*S; the
 * depot is at (0, 0).  W must be even.  Location id loc = (a*2+side)*L + k.
 *
 * Parity pins: see the module docstring of oracle/__init__.py; every function
 * here is pinned by at least one independent check in tests/.
 */
#ifndef WH_ORACLE_H
#define WH_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t n_aisles;          /* A */
    int32_t slots_per_side;    /* L */
    int32_t aisle_pitch;       /* P */
    int32_t slot_pitch;        /* S */
    int32_t cross_aisle_width; /* W (even) */
} or_layout;

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_ERANGE (-2)
#define OR_ENOMEM (-3)

/* Grid distance between (a1,y1) and (a2,y2): same aisle |y1-y2|, otherwise
 * P*|a1-a2| + min(y1+y2, 2Y-y1-y2). */
int64_t or_dist(const or_layout *g, int32_t a1, int32_t y1, int32_t a2, int32_t y2);

/* Tour lengths for a multiset of location ids (duplicates collapse).  A
 * negative return is an error code. */
int64_t or_sshape_tour(const or_layout *g, const int32_t *locs, int32_t n);
int64_t or_rr_tour(const or_layout *g, const int32_t *locs, int32_t n);
int64_t or_heldkarp_tour(const or_layout *g, const int32_t *locs, int32_t n);   /* <= 20 distinct */
int64_t or_permutation_tour(const or_layout *g, const int32_t *locs, int32_t n); /* <= 10 distinct */

/* Plan evaluation: tours of orders, orders of lines (SKUs), SKUs to
 * locations by slot_map + p*slot_map_stride (stride 0: one shared slotting).
 * Outputs may be NULL.  Returns OR_OK or an error. */
int or_eval_plans(const or_layout *g, int32_t n_orders, const int32_t *order_off,
                  const int32_t *line_sku, int32_t n_sku, const int32_t *slot_map,
                  int64_t slot_map_stride, int32_t n_plans, const int32_t *plan_tour_off,
                  const int32_t *tour_off, const int32_t *order_seq, int32_t *tour_s,
                  int32_t *tour_rr, int64_t *plan_s, int64_t *plan_rr);

/* Neighbourhood moves (Sec. 5: subroutine 4 evaluates a change in product
 * position; the picking list decides which orders are picked together).
 * moves[4*m .. 4*m+3] = {type, a, b, plan}:
 *   type 0: swap orders a and b between their tours of `plan`,
 *   type 1: relocate order a into tour b of `plan` (b local to the plan),
 *   type 2: swap the locations of SKUs a and b in `plan`'s slotting
 *           (per-plan slottings only, slot_map_stride > 0);
 *   type 3: relocate SKU a to location b, which must be empty in `plan`'s
 *           slotting (no SKU maps to it; subroutine 4 of Sec. 5 weighs moves
 *           into available empty places; per-plan slottings only).
 * Each move is applied to a copy of its plan, the whole plan is evaluated
 * before and after, and delta[2m], delta[2m+1] = (after - before) for the
 * S-shape and optimal rule.  status[m]: 0 applied, 1 infeasible (a changed
 * tour would exceed max_orders orders or max_lines lines; 0 = no cap),
 * 2 no-op (same tour, same SKU, or the SKU already at b), 3 invalid (id out
 * of range, order not in the plan, SKU move under a shared slotting, target
 * location occupied).  Deltas are 0 unless the
 * status is 0. */
int or_eval_moves(const or_layout *g, int32_t n_orders, const int32_t *order_off,
                  const int32_t *line_sku, int32_t n_sku, const int32_t *slot_map,
                  int64_t slot_map_stride, int32_t n_plans, const int32_t *plan_tour_off,
                  const int32_t *tour_off, const int32_t *order_seq, const int32_t *moves,
                  int32_t n_moves, int32_t max_orders, int32_t max_lines, int64_t *delta,
                  int32_t *status);

/* One best-improvement local-search step on every plan: plan p owns moves
 * [p*moves_per_plan, (p+1)*moves_per_plan) (their plan field must be p);
 * among those with status 0 and a negative optimal-cost delta the most
 * negative is applied, ties to the lowest index; applied[p] = that index
 * within the plan or -1.  The plans are edited in place: an order swap
 * exchanges the two entries of order_seq, a relocation removes the order from
 * its tour and appends it to the end of the target tour (tour_off shifts
 * between them), a SKU swap exchanges two entries of the plan's slotting, a
 * relocation sets the SKU's entry to the new location. */
int or_ls_step(const or_layout *g, int32_t n_orders, const int32_t *order_off, const int32_t *line_sku,
               int32_t n_sku, int32_t *slot_map, int64_t slot_map_stride, int32_t n_plans,
               const int32_t *plan_tour_off, int32_t *tour_off, int32_t *order_seq, const int32_t *moves,
               int32_t moves_per_plan, int32_t max_orders, int32_t max_lines, int32_t *applied);

/* ------------------------------------------------------- batch formation
 * Seed-and-grow batching of orders into picker tours (the paper's
 * clustering of orders and suggestion of which orders are picked together,
 * Sec. 5 and Sec. 6), scored by the exact optimal route length:
 *   seed  - the unassigned order whose tour alone is longest (ties: lowest id);
 *   grow  - while the tour holds fewer than max_orders orders (0: no cap), add
 *           the unassigned order whose lines fit (lines of the tour + its
 *           lines <= max_lines; 0: no cap) and that lengthens the tour least
 *           (ties: lowest id); stop when none fits;
 * until every order is in a tour.  Tours are emitted in order of formation,
 * the orders of a tour in order of insertion: tour_off [n_orders + 1] and
 * order_seq [n_orders] (a plan's CSR); *n_tours receives the tour count.
 * SKUs to locations by slot_map.  Returns OR_OK or an error. */
int or_batch_grow(const or_layout *g, int32_t n_orders, const int32_t *order_off, const int32_t *line_sku,
                  int32_t n_sku, const int32_t *slot_map, int32_t max_orders, int32_t max_lines,
                  int32_t *tour_off, int32_t *order_seq, int32_t *n_tours);

/* ------------------------------------------------------------ K-means slotting
 * Subproblem 3 (Sec. 5): products are placed by picking frequency, and an
 * unsupervised K-means classification (MacQueen 1967) decides which are
 * stored together; subroutine 4 scores the placement.  The paper gives no
 * features, initialisation or zone rule; the reading, all in integers:
 *   1. freq_s = lines of SKU s; co_s[j] = sum over every line of s and every
 *      OTHER line of the same order of signs[sku of that line][j] (the SKU's
 *      co-occurrence row projected on OR_KM_SKETCH random +-1 directions,
 *      signs [n_sku][OR_KM_DIM], column OR_KM_SKETCH unused).
 *   2. x_s[j] = trunc(co_s[j] * OR_KM_SCALE / n_s), n_s = floor(sqrt(sum co_s^2))
 *      (0 when n_s = 0) for j < OR_KM_SKETCH; x_s[OR_KM_SKETCH] =
 *      freq_weight * bitlen(freq_s) (bitlen(0) = 0, else floor(log2) + 1).
 *   3. centroid c = x of SKU init[c]; with init NULL, K-means++ seeding
 *      (Arthur & Vassilvitskii 2007) in integers from the caller's draws
 *      u[0..k): the first SKU is u[0] mod n_sku; with D(s) the squared
 *      distance from x_s to the nearest SKU chosen so far and T = sum D, the
 *      next is the first s (in id order) whose running sum D(0) + .. + D(s)
 *      exceeds u[c] mod T (u[c] mod n_sku when T = 0).
 *   4. iters Lloyd rounds: each SKU to its nearest centroid (squared
 *      Euclidean, ties to the lowest cluster); each non-empty cluster's
 *      centroid to floor((2 * sum + n) / (2 * n)) per coordinate (the mean
 *      rounded to the nearest integer, halves up); empty clusters keep theirs.
 *   5. a final assignment against the final centroids; weight of a cluster =
 *      the picks (freq) of its members.
 *   6. clusters ranked by weight (heavier first, ties lowest id); SKUs ordered
 *      by (cluster rank, freq descending, id).
 *   7. the r-th SKU of that order takes the r-th location in aisle-major order
 *      (aisle, then depth from the front, then side): r -> aisle r / 2L,
 *      depth (r mod 2L) / 2, side r mod 2.  Needs n_sku <= n_locations.
 * centroids [k][OR_KM_DIM], assign [n_sku], slot_map [n_sku]; x_out
 * [n_sku][OR_KM_DIM] and init_out [k] (the seeds used) may be NULL.
 * Returns OR_OK or an error. */
#define OR_KM_DIM 32
#define OR_KM_SKETCH 31
#define OR_KM_SCALE 1024
#define OR_KM_MAX_FREQ_WEIGHT 256
int or_kmeans_features(int32_t n_orders, const int32_t *order_off, const int32_t *line_sku, int32_t n_sku,
                       const int8_t *signs, int32_t freq_weight, int32_t *x, int32_t *freq);
int or_kmeans_pp_init(const int32_t *x, int32_t n, int32_t k, const uint64_t *u, int32_t *init);
/* step 4 and the final assignment of step 5 on rows x [n][OR_KM_DIM]:
 * centroids [k][OR_KM_DIM] holds the initial centroids on entry and the final
 * ones on return; assign [n] the final assignment. */
int or_kmeans_lloyd(const int32_t *x, int32_t n, int32_t k, int32_t iters, int32_t *centroids, int32_t *assign);
int or_kmeans_slotting(const or_layout *g, int32_t n_orders, const int32_t *order_off, const int32_t *line_sku,
                       int32_t n_sku, const int8_t *signs, int32_t freq_weight, int32_t k, const int32_t *init,
                       const uint64_t *u, int32_t iters, int32_t *x_out, int32_t *init_out, int32_t *centroids,
                       int32_t *assign, int32_t *slot_map);

/* ------------------------------------------------------------- surrogate
 * Learned prescreen (the paper's machine-learning-in-the-loop idea, Sec. 1 and
 * Fig. 1): a small MLP predicts a tour's normalised optimal length from a
 * fixed feature vector of the tour.
 *
 * Features, 192 per tour (the readings are listed in the design notes):
 *   [0, 64)    histogram over the visited aisles of their deepest pick,
 *              bin = floor(k_max * 64 / L) of the slot index;
 *   [64, 128)  the same for the shallowest pick (k_min);
 *   [128]      leftmost visited aisle * inv_A, [129] rightmost * inv_A,
 *   [130]      visited-aisle count * inv_A, [131] line count * (1/64);
 *   [132, 192) histogram of the visited aisles, bin = floor(a * 60 / A).
 * inv_A = (float)(1.0 / A).  Products are single-precision, as on the device;
 * all values are then representable or rounded to bf16 by the caller. */
int or_features(const or_layout *g, const int32_t *locs, int32_t n, float *out);

/* round a float to bfloat16 (round to nearest even), returned as float */
float or_bf16(float x);

/* MLP 192 -> 256 -> GELU -> 256 -> GELU -> 1.  Weights are given as floats
 * that are already bf16 values (w1[192*256] row-major [in][out], b1[256],
 * w2[256*256], b2[256], w3[256], b3[1]).  X is [n][192] of bf16 values.
 * Accumulation in double; each hidden activation is rounded to bf16 after
 * bias + GELU (0.5 x (1 + erf(x / sqrt 2))), as the device stores it.
 * y[n] receives the outputs (no rounding). */
void or_mlp_forward(const float *w1, const float *b1, const float *w2, const float *b2, const float *w3,
                    const float *b3, const float *X, int32_t n, double *y);

/* Loss 0.5 * mean((y - t)^2) and its gradient with respect to every
 * parameter (double), by the chain rule through the same forward pass with
 * the bf16 rounding points treated as identity. */
double or_mlp_backward(const float *w1, const float *b1, const float *w2, const float *b2, const float *w3,
                       const float *b3, const float *X, const double *t, int32_t n, double *g1, double *gb1,
                       double *g2, double *gb2, double *g3, double *gb3);

/* One training step with every intermediate kept ([n][256] row-major unless
 * noted): pre-activations z1, z2 and bf16 activations h1, h2 as in
 * or_mlp_forward; outputs y[n]; dy[n] = (y - t) / n; d2pre = dy * w3 *
 * gelu'(z2) and d2 = bf16(d2pre); s1 = d2 W2^T; d1pre = s1 * gelu'(z1) and
 * d1 = bf16(d1pre).  The back-propagated gradients are rounded to bf16 where
 * they become operands of a product (the bf16-operand contract of the
 * tensor-core training step); gradients g* as in or_mlp_backward but from
 * the rounded d2, d1.  Returns the loss 0.5 * mean((y - t)^2). */
double or_mlp_train_trace(const float *w1, const float *b1, const float *w2, const float *b2, const float *w3,
                          const float *b3, const float *X, const double *t, int32_t n, double *z1, double *h1,
                          double *z2, double *h2, double *y, double *dy, double *d2pre, double *d2, double *s1,
                          double *d1pre, double *d1, double *g1, double *gb1, double *g2, double *gb2, double *g3,
                          double *gb3);

/* One Adam step (Kingma & Ba 2015) on n parameters: m = b1 m + (1-b1) g,
 * v = b2 v + (1-b2) g^2, p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps). */
void or_adam(double *p, double *m, double *v, const double *g, int64_t n, double lr, double b1, double b2,
             double eps, int32_t step);

#ifdef __cplusplus
}
#endif
#endif
