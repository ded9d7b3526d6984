/*
 * wh.h -- C ABI of the GB300 warehouse order-picking plan evaluator.
 *
 * The library scores candidate order-picking plans for a single-block
 * rectangular warehouse: parallel aisles, a front and a back cross-aisle, and
 * the depot at the front end of aisle 0.  A plan is a SKU-to-location slotting
 * (product position x, Sec. 5, subproblem 3) plus a partition of the day's
 * orders (order history o, Sec. 5) into picker tours (the picking list,
 * Sec. 5, subroutine 5).  A tour's length is the picker's travel distance
 * (Sec. 5, subproblem 2, Eq. (2): min sum d_i), under two routing rules:
 *   - S-shape: every aisle holding a pick is traversed completely, alternating
 *     direction; with an odd number of such aisles the last one is entered and
 *     left from the front;
 *   - optimal: the shortest closed walk from the depot through all picks (the
 *     paper's Dijkstra distances and best picking sequence), computed exactly
 *     by the Ratliff-Rosenthal aisle-by-aisle dynamic programme.
 * A plan's cost is the int64 sum of its tours' int32 lengths (Eq. (2)).
 *
 * Geometry in integer units: aisle a has its centreline at x = a*aisle_pitch;
 * slot k (0 <= k < slots_per_side, either side of the aisle) lies at depth
 * cross_aisle_width/2 + k*slot_pitch; the front cross-aisle centre is depth 0,
 * the back one depth Y = cross_aisle_width + (slots_per_side-1)*slot_pitch.
 * Location ids: loc = (aisle*2 + side)*slots_per_side + k.
 *
 * Conventions shared by every call:
 *   - Return value: WH_OK (0) or a negative WH_E* code.  No exception or
 *     abort crosses the ABI.  Argument checks that need no device data run
 *     on the host before anything is launched; a failing call launches nothing.
 *   - Device pointers are CUDA device (or managed) addresses on the device
 *     that was current when the call was made.  Inputs and outputs are owned by
 *     the caller; the library owns only the layout handle and its scratch.
 *   - Work is enqueued on `stream` (a cudaStream_t passed as void*, NULL = the
 *     legacy default stream) and runs asynchronously.  Errors found on the
 *     device (an id out of range, a malformed offset array, a tour longer than
 *     WH_MAX_TOUR_LINES) set bits in a device status word that
 *     wh_get_last_status reads; the affected tours get cost -1 and are left out
 *     of their plan's sum.
 *   - One handle may be used from one host thread at a time; calls on the
 *     same handle from different streams must not overlap on the device.
 */
#ifndef WH_H
#define WH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define WH_OK 0
#define WH_EINVAL (-1)   /* bad argument: NULL pointer, negative size, bad mask */
#define WH_ERANGE (-2)   /* size beyond a documented limit, or an id out of range */
#define WH_ENOMEM (-3)   /* scratch allocation failed */
#define WH_ECUDA (-4)    /* a CUDA runtime call or launch failed */
#define WH_ETIMEOUT (-5) /* a bounded device-side wait gave up */

/* routing_mask bits */
#define WH_ROUTE_SSHAPE 1u
#define WH_ROUTE_OPTIMAL 2u

/* device status word bits (wh_get_last_status) */
#define WH_STATUS_BAD_ORDER 1u    /* order id outside [0, n_orders) */
#define WH_STATUS_BAD_SKU 2u      /* SKU id outside [0, n_sku) */
#define WH_STATUS_BAD_LOC 4u      /* slot_map entry outside [0, n_locations) */
#define WH_STATUS_BAD_OFFSET 8u   /* offsets decreasing or past the end of their array */
#define WH_STATUS_TOUR_TOO_LONG 16u
#define WH_STATUS_LONG_OVERFLOW 32u /* more long tours in one call than the deferral list holds */
#define WH_STATUS_TIMEOUT 64u       /* a bounded wait inside a kernel gave up (the kernel returned early) */

/* Limits of this implementation. */
#define WH_MAX_AISLES 65534
#define WH_MAX_SLOTS_PER_SIDE 65535
#define WH_MAX_TOUR_LINES 2048
/* 2*x_{A-1} + A*Y (the longest S-shape tour) must stay below this bound so the
 * device DP has int32 headroom for its partial costs. */
#define WH_MAX_TOUR_SPAN (1 << 27)

/* Warehouse geometry (Sec. 5: the design variable a, distance between racks,
 * is the aisle pitch here).  cross_aisle_width must be even and >= 2; all
 * other fields >= 1. */
typedef struct wh_layout_desc {
    int32_t n_aisles;
    int32_t slots_per_side;
    int32_t aisle_pitch;
    int32_t slot_pitch;
    int32_t cross_aisle_width;
} wh_layout_desc;

/* Opaque handle: the geometry plus the library's device scratch. */
typedef struct wh_layout wh_layout;

/* The day's order book (order history o, Sec. 5) in CSR form, device memory:
 * order o holds lines order_off[o] .. order_off[o+1]-1, line l asks for SKU
 * line_sku[l] in [0, n_sku).  order_off[0] must be 0 and order_off[n_orders]
 * equal n_lines. */
typedef struct wh_orders {
    int32_t n_orders;
    int32_t n_lines;
    int32_t n_sku;
    const int32_t *order_off; /* [n_orders + 1] */
    const int32_t *line_sku;  /* [n_lines] */
} wh_orders;

/* Candidate plans, device memory.  Slotting (product position x, Sec. 5):
 * SKU s of plan p sits at location slot_map[p*slot_map_stride + s];
 * slot_map_stride = 0 shares one slotting among all plans, otherwise it must be
 * >= n_sku.  Batching (picking lists, Sec. 5): plan p owns tours
 * plan_tour_off[p] .. plan_tour_off[p+1]-1 (global tour ids, plan_tour_off[0]
 * = 0, plan_tour_off[n_plans] = n_tours); tour t picks the orders
 * order_seq[tour_off[t] .. tour_off[t+1]-1] (tour_off[n_tours] <= n_seq).  A
 * tour's pick set is the set of locations of all lines of its orders
 * (repeats collapse); an empty tour costs 0. */
typedef struct wh_plans {
    int32_t n_plans;
    int32_t n_tours;
    int64_t n_seq;
    const int32_t *slot_map;
    int64_t slot_map_stride;
    const int32_t *plan_tour_off; /* [n_plans + 1] */
    const int32_t *tour_off;      /* [n_tours + 1] */
    const int32_t *order_seq;     /* [n_seq] */
    /* Optional (may be NULL): per-plan location occupancy, bit (l & 31) of
     * word p * ceil(n_locations / 32) + l / 32 set when a SKU of plan p sits
     * at location l.  Needed only by relocation moves (wh_eval_moves type 3),
     * built by wh_occupancy and kept current by wh_ls_apply. */
    uint32_t *loc_used;
} wh_plans;

/* Outputs, caller-owned device memory; any pointer may be NULL to skip it.
 * tour_* are per tour [n_tours] (int32), plan_* per plan [n_plans] (int64). */
typedef struct wh_costs {
    int32_t *tour_s;
    int32_t *tour_rr;
    int64_t *plan_s;
    int64_t *plan_rr;
} wh_costs;

/* Create a layout handle for the geometry `desc` (Sec. 5, Eq. (1)'s design
 * variable a and the rack layout of subsystem 1).  Host only: allocates the
 * handle, no device memory yet.  Returns WH_EINVAL for a NULL argument or a
 * non-positive / odd field, WH_ERANGE beyond WH_MAX_AISLES,
 * WH_MAX_SLOTS_PER_SIDE or WH_MAX_TOUR_SPAN.  *out is set only on success and
 * must be released with wh_destroy. */
int wh_create_layout(const wh_layout_desc *desc, wh_layout **out);

/* Score every tour and plan (Sec. 5, Eq. (2): sum over tours of d_i) under
 * the routing rules in routing_mask (WH_ROUTE_SSHAPE | WH_ROUTE_OPTIMAL, at
 * least one).  Costs are exact integers: int32 per tour, int64 per plan.
 * The first call on a device (or one with more lines / tours than any before)
 * allocates scratch with cudaMalloc, which synchronises; later calls allocate
 * nothing.  Returns WH_EINVAL (NULL handle/struct/pointer needed by the mask,
 * negative count, bad mask or stride), WH_ENOMEM, WH_ECUDA, or WH_OK once the
 * work is enqueued on `stream`. */
int wh_eval_plans(wh_layout *layout, const wh_orders *orders, const wh_plans *plans,
                  uint32_t routing_mask, const wh_costs *out, void *stream);

/* Neighbourhood moves for plan-level local search (Sec. 5: subroutine 4
 * evaluates a change in product position; the picking list decides which
 * orders are picked together).  moves[4*m .. 4*m+3] = {type, a, b, plan}:
 *   type 0: swap orders a and b between their tours of `plan`;
 *   type 1: relocate order a into tour b of `plan` (b counted from the
 *           plan's first tour);
 *   type 2: swap the locations of SKUs a and b in `plan`'s slotting (only
 *           with per-plan slottings, slot_map_stride > 0);
 *   type 3: relocate SKU a to location b, which must be empty in `plan`'s
 *           slotting (subroutine 4 weighs moves into available empty places;
 *           per-plan slottings and plans->loc_used, see wh_occupancy).
 * delta[2m], delta[2m+1] receive (after - before) of the plan's S-shape and
 * optimal cost; only the tours the move changes are re-costed, against their
 * current costs tour_s / tour_rr (the wh_eval_plans output for `plans`).
 * status[m]: 0 evaluated, 1 infeasible (a changed tour would exceed
 * max_orders_per_tour orders or max_lines_per_tour lines; 0 = no cap), 2 no-op
 * (same tour, same SKU, SKU already at the target), 3 invalid (id out of
 * range, order not in the plan, SKU move under a shared slotting, relocation
 * onto an occupied location or without loc_used, or a malformed tour); deltas are 0 unless
 * the status is 0.  Each plan must hold every order at most once.
 * All arrays are device memory.  The call synchronises `stream` twice (to
 * size its task list, then the record matrix of the tasks of more than 64
 * lines) and may allocate scratch.  Returns WH_OK, WH_EINVAL, WH_ENOMEM
 * or WH_ECUDA. */
int wh_eval_moves(wh_layout *layout, const wh_orders *orders, const wh_plans *plans, const int32_t *tour_s,
                  const int32_t *tour_rr, const int32_t *moves, int32_t n_moves, int32_t max_orders_per_tour,
                  int32_t max_lines_per_tour, int64_t *delta, int32_t *status, void *stream);

/* One step of best-improvement local search on every plan (Sec. 5: the
 * picking list and product positions are improved by evaluated moves).  Plan
 * p owns moves [p*moves_per_plan, (p+1)*moves_per_plan) (plan field p,
 * moves_per_plan <= 256) with their delta / status from wh_eval_moves; the
 * move with the most negative optimal-cost delta among those of status 0 and
 * negative delta is applied, ties to the lowest index; applied[p] receives its
 * index within the plan or -1.  The plans are edited IN PLACE (the const
 * pointers of `plans` are written): an order swap exchanges two entries of
 * order_seq; a relocation removes the order from its tour and appends it to
 * the end of the target tour, shifting order_seq and tour_off between them; a
 * SKU swap exchanges two entries of the plan's slotting; a relocation sets the
 * SKU's entry and, with plans->loc_used, moves its occupancy bit.  costs (may be NULL):
 * the plans' current per-tour and per-plan costs, updated in place for the
 * applied moves from the new tour costs that the wh_eval_moves (or
 * wh_surrogate_screen_eval) call which scored exactly these moves (same
 * `moves` pointer, the last move evaluation on this handle) computed -- no
 * full re-evaluation is needed; when NULL the
 * costs are left stale (refresh them with wh_eval_plans).  tour_changed (device,
 * one byte per tour, may be NULL; needs costs): set to 1 for every tour an
 * applied move rewrote, for wh_surrogate_screen's prediction cache; other
 * bytes are left as they are.  Each plan's segment of order_seq
 * may hold at most max(n_orders, 1) entries (WH_STATUS_BAD_OFFSET otherwise,
 * and that plan is left unchanged).  Returns WH_OK, WH_EINVAL, WH_ERANGE
 * (n_orders beyond 50,000: the staging buffer) or WH_ECUDA. */
int wh_ls_apply(wh_layout *layout, const wh_orders *orders, const wh_plans *plans, const int32_t *moves,
                int32_t moves_per_plan, const int64_t *delta, const int32_t *status, int32_t *applied,
                const wh_costs *costs, uint8_t *tour_changed, void *stream);

/* Occupancy bits of every plan's slotting, for relocation moves: writes
 * plans->loc_used (device, caller-owned, n_plans * ceil(n_locations / 32)
 * words) with bit l of plan p set when some SKU of plan p sits at location l.
 * Needs per-plan slottings (slot_map_stride > 0).  wh_ls_apply keeps the bits
 * current as it applies relocations.  Asynchronous on `stream`; allocates
 * nothing.  Returns WH_OK, WH_EINVAL or WH_ECUDA. */
int wh_occupancy(wh_layout *layout, const wh_orders *orders, const wh_plans *plans, void *stream);

/* Batch formation (Sec. 5 and Sec. 6: clustering the orders and suggesting
 * which orders are picked together): for each of n_maps slottings
 * (slot_map + p * slot_map_stride; stride 0: one shared slotting), partition
 * the orders into tours by seed and grow, scored by the exact optimal route
 * length:
 *   seed - the unassigned order whose tour alone is longest (ties: lowest id);
 *   grow - while the tour holds fewer than max_orders orders (0: no cap), add
 *          the unassigned order whose lines fit (tour lines + its lines <=
 *          max_lines; 0: no cap) and that lengthens the tour least (ties:
 *          lowest id); stop when none fits;
 * until every order is in a tour.  Outputs (device, caller-owned), per
 * slotting p: tour_off[p * (n_orders + 1) ...] (tour offsets into order_seq),
 * order_seq[p * n_orders ...] (tours in order of formation, orders in order
 * of insertion), n_tours[p] (-1 when the slotting maps a line outside the
 * layout: status bit WH_STATUS_BAD_LOC).  Needs A <= 255, L <= 256 and
 * n_orders <= 65,535 (WH_ERANGE otherwise) and the
 * order book in shared memory (about 12 B per order + 2 B per line + 38 B per
 * aisle <= 200 KB, WH_ERANGE otherwise).  Asynchronous on `stream`; allocates
 * nothing.  Returns WH_OK, WH_EINVAL, WH_ERANGE or WH_ECUDA. */
int wh_batch_grow(wh_layout *layout, const wh_orders *orders, const int32_t *slot_map, int64_t slot_map_stride,
                  int32_t n_maps, int32_t max_orders, int32_t max_lines, int32_t *tour_off, int32_t *order_seq,
                  int32_t *n_tours, void *stream);

/* K-means slotting (Sec. 5, subproblem 3: products placed by picking
 * frequency, an unsupervised K-means classification (MacQueen 1967) deciding
 * which are stored together; subroutine 4 scores the placement with
 * wh_eval_plans).  The paper fixes no features, seeding or zone rule; this is
 * the library's reading, all in integers (so the result is exact):
 *   1. freq_s = lines of SKU s; co_s[j] = sum over every line of s and every
 *      OTHER line of the same order of signs[that line's SKU][j], j < 31 (the
 *      SKU's co-occurrence row projected on 31 random +-1 directions);
 *   2. x_s[j] = trunc(co_s[j] * 1024 / floor(sqrt(sum co_s^2))) (0 when the
 *      root is 0), j < 31; x_s[31] = freq_weight * bitlen(freq_s);
 *   3. seeds: init[0..k) when init is non-NULL, else K-means++ (Arthur &
 *      Vassilvitskii 2007) from the draws u[0..k): seed 0 = u[0] mod n_sku,
 *      seed c = the first SKU whose running sum of D^2 (squared distance to
 *      the nearest seed so far, in SKU order) exceeds u[c] mod sum D^2
 *      (u[c] mod n_sku when that sum is 0); centroid c = x of seed c;
 *   4. iters Lloyd rounds: nearest centroid (squared Euclidean, ties to the
 *      lowest cluster), then every non-empty centroid = floor((2 * sum + n) /
 *      (2 * n)) per coordinate (the mean, rounded to nearest, halves up);
 *   5. a final assignment; a cluster's weight = the picks of its members;
 *   6. clusters ranked by weight (heavier first, ties lowest id), SKUs by
 *      (cluster rank, picks descending, id); the r-th SKU takes the r-th
 *      location in aisle-major order: aisle r / 2L, depth index (r mod 2L) / 2,
 *      side r mod 2 (locations past n_sku stay empty).
 * Inputs (device): signs int8 [n_sku][32] of +-1 (column 31 unused; 16-byte
 * aligned); init int32 [k] or NULL; u uint64 [k] (needed when init is NULL).
 * Outputs (device, caller-owned): centroids int32 [k][32], assign int32
 * [n_sku], slot_map int32 [n_sku] (a slotting for wh_plans.slot_map);
 * optional x_out int32 [n_sku][32] (16-byte aligned) and init_out int32 [k]
 * (the seeds used).  Needs 1 <= k <= min(256, n_sku), 0 <= freq_weight <= 256,
 * iters >= 0, n_sku <= the layout's locations and n_lines < 2^26 (WH_EINVAL
 * or WH_ERANGE otherwise).  A SKU id or seed outside [0, n_sku) sets
 * WH_STATUS_BAD_SKU, bad order offsets WH_STATUS_BAD_OFFSET (the outputs are
 * then unspecified).  Asynchronous on `stream`; uses the handle's scratch
 * (about 400 B per SKU), growing it when needed.  Returns WH_OK, WH_EINVAL,
 * WH_ERANGE, WH_ENOMEM or WH_ECUDA. */
int wh_kmeans_slotting(wh_layout *layout, const wh_orders *orders, const int8_t *signs, int32_t freq_weight,
                       int32_t k, const int32_t *init, const uint64_t *u, int32_t iters, int32_t *x_out,
                       int32_t *init_out, int32_t *centroids, int32_t *assign, int32_t *slot_map, void *stream);

/* Explicit optimal routes (Sec. 5, Eq. (2): the picking route of a tour is
 * the best order of its picking positions, shortest paths between them; Sec.
 * 6 hands the picker that sequence).  For each of the n listed tours
 * (tours[i]: a global tour index into plans->tour_off; the tour's plan, for
 * per-plan slottings, is found from plan_tour_off), write its distinct pick
 * points in visiting order along an optimal closed walk from the depot,
 * obtained from the Ratliff-Rosenthal DP's decisions (Ratliff & Rosenthal,
 * Oper. Res. 31(3), 1983) and an Euler circuit of the route subgraph they
 * fix.  A pick point is aisle << 16 | slot index: the two sides of an aisle
 * at one depth are one point.  Outputs (device, caller-owned):
 * points[i * max_points ...] (int32, n_points[i] entries used),
 * n_points[i] (-1 on error), length[i] (the route's length, which equals the
 * optimal tour length; -1 on error).  Walking the points in order with
 * shortest paths between consecutive ones, from and back to the depot,
 * covers exactly length[i].  A tour with more than min(max_points, 256)
 * distinct points sets WH_STATUS_TOUR_TOO_LONG; a bad tour index or offsets
 * WH_STATUS_BAD_OFFSET; bad ids WH_STATUS_BAD_ORDER / WH_STATUS_BAD_LOC.  One
 * thread per tour, about 10 KB of local memory each; meant for the tours of
 * a chosen plan, not for scoring.  Asynchronous on `stream`; allocates
 * nothing.  Returns WH_OK, WH_EINVAL or WH_ECUDA. */
int wh_routes(wh_layout *layout, const wh_orders *orders, const wh_plans *plans, const int32_t *tours, int32_t n,
              int32_t max_points, int32_t *points, int32_t *n_points, int32_t *length, void *stream);

/* ------------------------------------------------------------------------
 * Learned prescreen (machine learning in the decision loop, Sec. 1 and
 * Fig. 1): an MLP 192 -> 256 -> GELU -> 256 -> GELU -> 1 predicts a tour's
 * optimal length divided by 2*x_{A-1} + A*Y from 192 tour features; bf16
 * weights and activations, fp32 accumulation, trained on the device with
 * Adam on fp32 master weights.  Parameters are one packed float vector of
 * WH_MLP_NPARAM values: w1 [192][256], b1 [256], w2 [256][256], b2 [256],
 * w3 [256], b3 [1] (row-major, [input][output]).
 */
#define WH_MLP_NPARAM 115457
#define WH_FEATURES 192

typedef struct wh_surrogate wh_surrogate;

/* Features of every tour of `plans` into X (device, bf16 stored as uint16,
 * [n_tours][192], rows 16-byte aligned): histograms over the tour's visited
 * aisles of the deepest and the shallowest pick's slot bin floor(k*64/L)
 * (features 0..63, 64..127), leftmost aisle / A, rightmost aisle / A,
 * visited-aisle count / A, line count / 64 (128..131), and a 60-bin
 * histogram of the visited aisles floor(a*60/A) (132..191).  Tours with more
 * than 128 distinct aisles set WH_STATUS_TOUR_TOO_LONG.  Returns WH_OK,
 * WH_EINVAL, WH_ERANGE (slots_per_side > 256), WH_ENOMEM or WH_ECUDA. */
int wh_surrogate_features(wh_layout *layout, const wh_orders *orders, const wh_plans *plans, uint16_t *X,
                          void *stream);

/* Create a surrogate on the current device: Xavier-uniform weights drawn
 * from `seed` (SplitMix64), zero biases, zero Adam state.  Allocates and
 * synchronises.  Returns WH_OK, WH_EINVAL, WH_ENOMEM or WH_ECUDA. */
int wh_surrogate_create(uint64_t seed, wh_surrogate **out);

/* Replace the parameters (host array of WH_MLP_NPARAM floats) and reset the
 * Adam state.  Synchronises. */
int wh_surrogate_set_params(wh_surrogate *s, const float *host_params);

/* Copy the fp32 master parameters and / or the last step's gradients to host
 * arrays of WH_MLP_NPARAM floats (either may be NULL).  Synchronises. */
int wh_surrogate_get_params(wh_surrogate *s, float *host_params, float *host_grads);

/* y[i] = MLP(X[i]) for n rows of bf16 features (device, row-major [n][192],
 * 16-byte aligned); fp32 outputs.  Runs on the tcgen05 tensor cores; its
 * bounded waits report WH_STATUS_TIMEOUT through wh_surrogate_get_status.
 * Allocates nothing.  Returns WH_OK, WH_EINVAL (NULL or misaligned X) or
 * WH_ECUDA. */
int wh_surrogate_predict(wh_surrogate *s, const uint16_t *X, int64_t n, float *y, void *stream);

/* Test of the prediction kernel's failure handling (no counterpart in the
 * paper): the same launch as wh_surrogate_predict, but the kernel's producer
 * stops before 128-row tile `skip_tile` (0 <= skip_tile < ceil(n / 128)) and
 * every barrier wait gives up after wait_ns nanoseconds (1,000 ..
 * 2,000,000,000).  The wait for that tile's features then runs out: the CTA
 * sets WH_STATUS_TIMEOUT in the surrogate's status word, its other roles leave
 * their loops, copies and MMAs in flight are waited for and the tensor memory
 * is freed, so the context stays usable; y is incomplete.  Read the status
 * with wh_surrogate_get_status.  Returns WH_OK, WH_EINVAL or WH_ECUDA. */
int wh_surrogate_predict_timeout_test(wh_surrogate *s, const uint16_t *X, int64_t n, float *y, int64_t skip_tile,
                                      uint64_t wait_ns, void *stream);

/* Read and clear the surrogate's device status word (WH_STATUS_* bits of the
 * prediction kernels).  Synchronises the device. */
int wh_surrogate_get_status(wh_surrogate *s, uint32_t *out);

/* One Adam step (lr; beta1 0.9, beta2 0.999, eps 1e-8) on the mean squared
 * error 0.5*mean((y - target)^2) of n rows; *loss_out (device float, may be
 * NULL) receives the loss before the step.  Allocates scratch when n grows. */
int wh_surrogate_train_step(wh_surrogate *s, const uint16_t *X, const float *target, int32_t n, float lr,
                            float *loss_out, void *stream);

/* Intermediates of the last wh_surrogate_train_step (a check of the
 * training step layer by layer against a reference; Sec. 1 / Fig. 1,
 * config 5's bf16 weights and activations with fp32 accumulation): copy the
 * first n_rows rows (n_rows <= that step's n) of one saved buffer to dst
 * (device, caller-owned), enqueued on `stream`:
 *   WH_TRACE_Z1, WH_TRACE_Z2   fp32 [n_rows][256] pre-activations;
 *   WH_TRACE_H1, WH_TRACE_H2   bf16 [n_rows][256] activations;
 *   WH_TRACE_Y, WH_TRACE_DY    fp32 [n_rows] outputs and (y - target) / n;
 *   WH_TRACE_DZ2, WH_TRACE_DZ1 bf16 [n_rows][256] back-propagated gradients
 *                              of the pre-activations (the backward GEMMs'
 *                              operands).
 * The buffers hold the last step's values until the next training step.
 * Returns WH_OK or WH_EINVAL (unknown buffer, rows beyond the last step). */
#define WH_TRACE_Z1 0
#define WH_TRACE_H1 1
#define WH_TRACE_Z2 2
#define WH_TRACE_H2 3
#define WH_TRACE_Y 4
#define WH_TRACE_DY 5
#define WH_TRACE_DZ2 6
#define WH_TRACE_DZ1 7
int wh_surrogate_get_trace(wh_surrogate *s, int32_t which, void *dst, int64_t n_rows, void *stream);

/* Prescreen of local-search moves: for plan p's moves [p*moves_per_plan,
 * (p+1)*moves_per_plan) the surrogate predicts each move's change of the
 * plan's optimal cost (sum over the tours the move changes of predicted new
 * minus predicted current length) and keeps the `keep` moves with the lowest
 * prediction (ties: lowest index) in kept[(p*keep + j)*4 .. +3]; places
 * without an eligible move get {9, 0, 0, p}, which wh_eval_moves reports as
 * invalid.  Score the kept moves exactly with wh_eval_moves.
 * Prediction cache of the current tours (both may be NULL):
 *   y_tour_cache NULL: every tour is predicted, nothing kept;
 *   y_tour_cache set, tour_changed NULL: every tour is predicted into the
 *     cache (float per tour, device);
 *   both set: only the tours whose tour_changed byte is non-zero (as
 *     wh_ls_apply sets them) are predicted into the cache, and their bytes
 *     are cleared; the other entries must hold the current predictions.
 * Synchronises `stream` (once, twice with tour_changed); may allocate
 * scratch.  Returns WH_OK, WH_EINVAL, WH_ERANGE, WH_ENOMEM or WH_ECUDA. */
int wh_surrogate_screen(wh_layout *layout, wh_surrogate *s, const wh_orders *orders, const wh_plans *plans,
                        const int32_t *moves, int32_t moves_per_plan, int32_t keep, int32_t max_orders_per_tour,
                        int32_t max_lines_per_tour, float *y_tour_cache, uint8_t *tour_changed, int32_t *kept,
                        void *stream);

/* The prescreen of wh_surrogate_screen followed by the exact scores of the
 * kept moves, as one call: kept [n_plans * keep][4] as wh_surrogate_screen
 * writes it, and its move deltas kept_delta [n_plans * keep][2] (int64) and
 * statuses kept_status [n_plans * keep] (int32) exactly as wh_eval_moves on
 * `kept` with the current tour costs tour_s / tour_rr would give them.  The
 * exact pass reuses the prescreen's per-plan order -> tour table and SKU ->
 * orders index (the plans do not change inside the call) instead of building
 * them again.  The result feeds wh_ls_apply like that wh_eval_moves call would
 * (pass `kept` as its moves and `keep` as moves_per_plan).  Synchronises
 * `stream` as the two calls do.  Returns as wh_surrogate_screen, WH_EINVAL also
 * for a NULL tour_s, tour_rr, kept_delta or kept_status. */
int wh_surrogate_screen_eval(wh_layout *layout, wh_surrogate *s, const wh_orders *orders, const wh_plans *plans,
                             const int32_t *moves, int32_t moves_per_plan, int32_t keep,
                             int32_t max_orders_per_tour, int32_t max_lines_per_tour, float *y_tour_cache,
                             uint8_t *tour_changed, const int32_t *tour_s, const int32_t *tour_rr, int32_t *kept,
                             int64_t *kept_delta, int32_t *kept_status, void *stream);

/* Diagnostics of the last wh_surrogate_screen call on `layout` (device
 * pointers into the layout's scratch, valid until its next call; all NULL and
 * *n_tasks = 0 when the last call was not a screen): the number of tasks (one
 * per changed tour of a move: an order move has two, a SKU move one per order
 * holding a moved SKU), the task list [n_tasks][4] (move index, changed tour,
 * then order added / order removed for order moves or the order holding the
 * SKU / a tag for SKU moves), whether each task counts ([n_tasks][2] int32:
 * 0, 0 counted; -1, -1 not: invalid ids, or a SKU-swap task that another task
 * of the same tour stands for) and the bf16 feature rows of the changed tours
 * [n_tasks][192] that the screen predicted from (Sec. 1, Fig. 1).  Enqueues
 * nothing.  Returns WH_OK or WH_EINVAL. */
int wh_surrogate_screen_trace(wh_layout *layout, int64_t *n_tasks, const int32_t **tasks, const int32_t **counted,
                              const uint16_t **features);

void wh_surrogate_destroy(wh_surrogate *s);

/* Sizes accepted by wh_eval_plans_noalloc. */
#define WH_NOALLOC_MAX_LINES (1 << 20)
#define WH_NOALLOC_MAX_TOURS (1 << 20)

/* wh_eval_plans for callers that cannot allocate device memory (the paper has
 * no counterpart; this is an interface for embedding).  Some callers must not
 * let a library call cudaMalloc or cudaFree: a serving process whose device
 * memory is fully reserved up front by its own pool, where one more cudaMalloc
 * would fail or upset its memory plan, or a loop that cannot afford the
 * device-wide synchronisation that cudaMalloc / cudaFree may cause.  This call
 * takes the geometry directly (no handle) and computes exactly what
 * wh_eval_plans computes, with the same kernels, but its scratch lives in one
 * fixed device array inside the library (about 16 MiB, held on every GPU that
 * loads the library until the process exits); it allocates nothing.
 *   - Limits: orders->n_lines <= WH_NOALLOC_MAX_LINES and
 *     plans->n_tours <= WH_NOALLOC_MAX_TOURS, else WH_ERANGE before any work.
 *   - status: optional caller-owned device word; the call zeroes it on
 *     `stream` and the kernels OR WH_STATUS_* bits into it.  NULL: the bits
 *     go to a word inside the library's array, cleared by each call and
 *     reported nowhere (errors found on the device then show only as tour
 *     costs of -1).
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - Every call shares the one array: calls that may overlap on the GPU (on
 *     different streams, or from different threads) race and corrupt each
 *     other's results.  Serialise them.
 * Returns as wh_eval_plans (WH_EINVAL for a bad desc or argument). */
int wh_eval_plans_noalloc(const wh_layout_desc *desc, const wh_orders *orders, const wh_plans *plans,
                          uint32_t routing_mask, const wh_costs *out, uint32_t *status, void *stream);

/* ------------------------------------------------------------------------
 * Batched evaluation: many independent warehouse instances of uneven size
 * (each its own geometry, order book, shared slotting and plans) scored in
 * one persistent launch.  This is the paper's subsystem evaluation run for
 * many candidate designs at once (Sec. 4: subsystem work distributed to GPU
 * nodes; Sec. 5, Eq. (2) per instance).  The launch takes (instance, chunk
 * range) work items from a device queue ordered largest first; it can be
 * replayed as a CUDA graph.
 */
typedef struct wh_instance {
    wh_layout_desc layout;
    wh_orders orders;
    wh_plans plans;   /* slot_map_stride must be 0 (one slotting per instance) */
    wh_costs out;
    /* Optional (may be NULL): the plans' order ids as unsigned 16-bit values
     * [plans.n_seq] (device memory; needs orders.n_orders <= 65,536).  When
     * every instance of the batch sets it, the batch reads these instead of
     * plans.order_seq (which may then be NULL): half the bytes, and host-
     * resident plans cross the host link and are scored without a widening
     * pass.  Setting it on some instances and not others is WH_EINVAL. */
    const uint16_t *order_seq16;
} wh_instance;

typedef struct wh_batch wh_batch;

/* Validate n >= 1 instance descriptors (host array; the data they point to
 * is device memory, which must stay valid and unchanged in size while the
 * batch lives), copy them to the device and build the work queue.
 * Allocates device memory (synchronises).  Returns WH_OK, WH_EINVAL (an
 * instance fails the checks of wh_create_layout / wh_eval_plans, or uses
 * per-plan slottings), WH_ERANGE, WH_ENOMEM or WH_ECUDA. */
int wh_batch_create(const wh_instance *insts, int32_t n, wh_batch **out);

/* Launch shape: CTA size (32..384 with 16-bit keys, layouts of <= 255 aisles
 * and <= 256 slots per side; 32..256 otherwise; a multiple of 32), 32-tour chunks per work
 * item (>= 1) and whether order books are staged in shared memory (0/1; it
 * is turned off when the largest order book does not fit).  Rebuilds the
 * work queue and drops captured graphs.  Returns WH_OK or WH_EINVAL. */
int wh_batch_set_tuning(wh_batch *b, int32_t threads, int32_t chunks_per_item, int32_t smem_tables);

/* Read the launch shape in use. */
int wh_batch_get_tuning(wh_batch *b, int32_t *threads, int32_t *chunks_per_item, int32_t *smem_tables);

/* Score every tour and plan of every instance (as wh_eval_plans does for
 * one), enqueued on `stream`.  Returns WH_OK, WH_EINVAL or WH_ECUDA. */
int wh_batch_eval(wh_batch *b, uint32_t routing_mask, void *stream);

/* Same work, replayed from a CUDA graph that the first call for a given
 * routing_mask captures (on a private stream) and instantiates. */
int wh_batch_eval_graph(wh_batch *b, uint32_t routing_mask, void *stream);

/* Autotuner: time candidate launch shapes (CTA size 128, 256 or, with 16-bit
 * keys, 384 x 2 to 4,096 chunks of 32 tours per work item, powers of two,
 * and for 384 threads also 12 to 1,536 chunks, multiples of its 12 warps, which
 * split an item evenly over them) on this batch with the given mask, keep the
 * fastest and report it.  When
 * cache_path is not NULL the choice is looked up first, and stored after, in
 * that JSON file under a key built from the batch's size bucket (key width,
 * instance count, total tours, largest order book, mask).  Synchronises
 * `stream`.  Returns WH_OK, WH_EINVAL or WH_ECUDA. */
int wh_batch_autotune(wh_batch *b, uint32_t routing_mask, const char *cache_path, void *stream,
                      int32_t *threads, int32_t *chunks_per_item, int32_t *from_cache);

/* Read and clear the batch's device status word (WH_STATUS_* bits).
 * Synchronises `stream`. */
int wh_batch_get_status(wh_batch *b, void *stream, uint32_t *status);

/* Release the batch (device memory and graphs).  NULL is a no-op. */
void wh_batch_destroy(wh_batch *b);

/* Widen n unsigned 16-bit values to int32, device to device (src and dst
 * device memory, caller-owned, not overlapping).  Order ids fit 16 bits when
 * n_orders <= 65,536, so host-resident plans can cross the host link at half
 * the bytes and be widened on the device before wh_eval_plans.  Asynchronous
 * on `stream`; allocates nothing.  Returns WH_OK, WH_EINVAL or WH_ECUDA. */
int wh_widen_u16(const uint16_t *src, int32_t *dst, int64_t n, void *stream);

/* Read and clear the device status word of `layout` (WH_STATUS_* bits of all
 * calls since the last read).  Synchronises `stream`.  Returns WH_OK,
 * WH_EINVAL or WH_ECUDA. */
int wh_get_last_status(wh_layout *layout, void *stream, uint32_t *status);

/* Work of the last wh_eval_moves call on this handle (measurement aid; no
 * counterpart in the paper): *tours = changed tours walked (one per task of
 * the moves: the tours a move rewrites), *lines = their order lines.
 * Synchronises `stream`.  Returns WH_OK, WH_EINVAL or WH_ECUDA. */
int wh_get_move_stats(wh_layout *layout, void *stream, int64_t *tours, int64_t *lines);

/* Kernel timing of a batch (tracing aid; no counterpart in the paper), as
 * wh_set_timing / wh_get_timing for a layout: while enabled, every kernel that
 * wh_batch_eval launches (k_prep_batch, k_eval_batch, k_eval_long) is
 * bracketed by two CUDA events on the launch's stream.  Graph replays
 * (wh_batch_eval_graph) carry no events and are not counted.  Enabling
 * resets the totals.  Returns WH_OK, WH_EINVAL or WH_ECUDA. */
int wh_batch_set_timing(wh_batch *b, int enable);
int wh_batch_get_timing(wh_batch *b, int32_t *n_kernels, const char **names, int32_t *launches,
                        double *total_ms, int32_t cap);

/* Kernel timing (tracing aid; no counterpart in the paper).  While enabled,
 * every kernel this handle launches is bracketed by two CUDA events recorded
 * on the launch's stream; wh_get_timing synchronises on those events and
 * reports, per kernel name, the number of launches and their summed device
 * time since timing was enabled.  Enabling resets the totals.  Returns WH_OK,
 * WH_EINVAL or WH_ENOMEM. */
int wh_set_timing(wh_layout *layout, int enable);

/* Fill up to `cap` entries: names[i] (static strings owned by the library),
 * launches[i], total_ms[i]; *n_kernels receives the number of kernel kinds.
 * Returns WH_OK, WH_EINVAL or WH_ECUDA. */
int wh_get_timing(wh_layout *layout, int32_t *n_kernels, const char **names, int32_t *launches,
                  double *total_ms, int32_t cap);

/* Release the handle and its device scratch.  The caller must make sure no
 * work that uses the handle is still running.  NULL is a no-op. */
void wh_destroy(wh_layout *layout);

#ifdef __cplusplus
}
#endif
#endif
