// Plan evaluation kernels for sm_103a.
//
// What is computed (Sec. 5, Eq. (2)): for every tour, the length of the
// S-shape route and of the optimal route through its picks, and for every
// plan the int64 sum of its tours' lengths.
//
// Design (one GPU, integer work; nothing here is a dense contraction):
//   k_prep        -- layout / slot-map build: one packed key (aisle<<16 | slot)
//                    per order line under the shared slotting; zeroes the
//                    per-plan sums and the long-tour counter.
//   k_eval_short  -- one tour per thread for tours of <= 64 lines.  A warp
//                    owns 32 consecutive tours; keys are gathered from the
//                    shared-memory order book into registers and sorted by a
//                    fully unrolled bitonic network (two 16-bit keys per
//                    register when the layout allows, so one min/max pair
//                    serves two comparators), reduced to per-aisle records
//                    (aisle, shallowest and deepest pick, largest gap between
//                    consecutive picks) in shared memory, then the S-shape
//                    closed form and the optimal-route DP run over the
//                    records.  Plan sums: a segmented warp reduction and one
//                    int64 atomic per (warp, plan) segment; no CTA barrier
//                    after the table staging.
//   k_eval_long   -- one warp per tour for longer tours: shared-memory
//                    bitonic sort, then one lane runs the record scan and DP.
//
// The optimal-route DP is the Ratliff-Rosenthal programme in a reduced form:
// the depot is a_0 itself (start state "a_0 in the tour, even degree"), the
// classes (0,0,0C) and (0,0,1C) never need to be stored, and a run of aisles
// without picks is crossed in one step (every class keeps to the cheapest
// horizontal edge pattern it can use there), so the DP costs one step per
// aisle that holds a pick instead of one per aisle up to the rightmost pick.
#include <type_traits>

#include "tour_core.cuh"

namespace wh {

namespace {

// Per-instance staging of the order book into shared memory: one descriptor
// per order (first line << 8 | line count; count 255 marks an order that the
// short path does not take: malformed, or 255 lines or more, so its tours go
// to the long-tour kernel, which checks them) and one key (or SKU) per line.
// Loads are issued STAGE_BATCH at a time before their stores, so that each
// thread keeps that many global reads in flight.  Returns true when one of
// this thread's staged keys is the bad-key marker (a line whose SKU or slot is
// invalid) or when keys are not staged (per-plan slottings): the evaluation
// then checks every tour's keys.
constexpr int STAGE_BATCH = 8;

template <bool KEY16, bool SHARED_MAP>
__device__ __forceinline__ bool stage_tables(const EvalArgs& a, uint32_t* s_desc, void* s_tab, KeySrc& src,
                                             int tid, int T) {
    bool bad = false;
    for (int o0 = tid; o0 < a.n_orders; o0 += STAGE_BATCH * T) {
        int lbs[STAGE_BATCH], les[STAGE_BATCH];
#pragma unroll
        for (int u = 0; u < STAGE_BATCH; ++u) {
            const int o = o0 + u * T;
            lbs[u] = o < a.n_orders ? a.order_off[o] : 0;
            les[u] = o < a.n_orders ? a.order_off[o + 1] : 0;
        }
#pragma unroll
        for (int u = 0; u < STAGE_BATCH; ++u) {
            const int o = o0 + u * T;
            if (o >= a.n_orders) continue;
            const int lb = lbs[u], le = les[u];
            const bool ok = lb >= 0 && le >= lb && le <= a.n_lines && le - lb < 255 && lb < (1 << 24);
            s_desc[o] = ok ? ((uint32_t)lb << 8) | (uint32_t)(le - lb) : 0xFFu;
        }
    }
    if constexpr (SHARED_MAP) {
        if constexpr (KEY16) {
            uint16_t* k16 = static_cast<uint16_t*>(s_tab);
            for (int i0 = tid; i0 < a.n_lines; i0 += STAGE_BATCH * T) {
                uint32_t k[STAGE_BATCH];
#pragma unroll
                for (int u = 0; u < STAGE_BATCH; ++u) {
                    const int i = i0 + u * T;
                    k[u] = i < a.n_lines ? a.line_key[i] : 0u;
                }
#pragma unroll
                for (int u = 0; u < STAGE_BATCH; ++u) {
                    const int i = i0 + u * T;
                    if (i >= a.n_lines) continue;
                    const uint32_t k16v = key16_of(k[u]);
                    bad |= k16v == KEY16_BAD;
                    k16[i] = (uint16_t)k16v;
                }
            }
        } else {
            uint32_t* k32 = static_cast<uint32_t*>(s_tab);
            for (int i = tid; i < a.n_lines; i += T) {
                const uint32_t k = a.line_key[i];
                bad |= k == KEY_BAD;
                k32[i] = k;
            }
        }
        src.keys = s_tab;
    } else {
        int32_t* sk = static_cast<int32_t*>(s_tab);
        for (int i = tid; i < a.n_lines; i += T) sk[i] = a.line_sku[i];
        src.skus = sk;
        bad = true;
    }
    src.desc = s_desc;
    return bad;
}

__device__ __forceinline__ KeySrc global_src(const EvalArgs& a) {
    KeySrc src;
    src.off = a.order_off;
    src.desc = nullptr;
    src.keys = a.line_key;
    src.skus = a.line_sku;
    src.map = nullptr;
    return src;
}

// Defer tour t of plan `plan` (instance `inst`) to the long-tour kernel.
__device__ __forceinline__ bool defer_long(const EvalArgs& a, int inst, int t, int plan) {
    const int slot = atomicAdd(a.long_count, 1);
    if (slot >= a.long_cap) {
        flag(a.status, WH_STATUS_LONG_OVERFLOW);
        return false;
    }
    a.long_list[3 * slot] = inst;
    a.long_list[3 * slot + 1] = t;
    a.long_list[3 * slot + 2] = plan;
    return true;
}

// Order id at sequence position q: the 16-bit copy when ID16 (batched
// instances whose order books have at most 65,536 orders), else int32.
template <bool ID16>
__device__ __forceinline__ int order_id(const EvalArgs& a, int64_t q) {
    if constexpr (ID16) return (int)__ldg(reinterpret_cast<const unsigned short*>(a.order_seq16) + q);
    else return __ldg(a.order_seq + q);
}

// this warp's contiguous range of 32-tour chunks: chunks split evenly over
// all warps of the grid (each warp takes floor or ceil of chunks / warps,
// none is left without work while another takes an extra chunk)
__device__ __forceinline__ void warp_chunk_range(const EvalArgs& a, int& c_begin, int& c_end) {
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t n_chunks = ((int64_t)a.n_tours + 31) >> 5;
    c_begin = (int)(gw * n_chunks / warps);
    c_end = (int)((gw + 1) * n_chunks / warps);
}

// Plan of tour t0 (the largest p with plan_tour_off[p] <= t0), found by the
// whole warp: each round probes 32 evenly spaced offsets of the remaining
// range at once and keeps the piece between the last probe at or below t0
// and the next, so the range shrinks 32-fold per round (3 dependent loads
// for 4,096 plans instead of 12).  Every lane returns the same plan.
__device__ __forceinline__ int warp_find_plan(const EvalArgs& a, int t0, int lane) {
    int lo = 0, hi = a.n_plans - 1;
    while (lo < hi) {
        const int span = hi - lo;                         // candidates lo+1 .. hi
        const int idx = lo + (int)(((int64_t)span * (lane + 1) + 31) / 32);   // in [lo+1, hi], non-decreasing
        const bool le = a.plan_tour_off[idx] <= t0;
        const unsigned below = __ballot_sync(0xffffffffu, le);   // a prefix of the lanes
        const int k = __popc(below);
        const int lo_new = k ? __shfl_sync(0xffffffffu, idx, k - 1) : lo;
        const int hi_new = k < 32 ? __shfl_sync(0xffffffffu, idx, k < 32 ? k : 31) - 1 : hi;
        lo = lo_new;
        hi = hi_new;
    }
    return lo;
}

// One warp scores the 32-tour chunks [c_begin, c_end) of instance `a`, one
// tour per lane, and adds its plans' sums with one atomic per plan segment.
template <bool KEY16, bool SHARED_MAP, bool SMEM_TABLES, bool ID16 = false>
__device__ __forceinline__ void eval_chunks(const EvalArgs& a, KeySrc src, uint32_t mask, int inst, int c_begin,
                                            int c_end, uint32_t* col16, uint2* col32, int T, int lane,
                                            bool check_keys) {
    const bool need_rr = (mask & WH_ROUTE_OPTIMAL) != 0;
    const bool want_s = (mask & WH_ROUTE_SSHAPE) != 0;
    // staged order book (shared memory): descriptors and per-line keys
    uint32_t desc_sa = 0, keys_sa = 0;
    if constexpr (SMEM_TABLES) {
        desc_sa = smem_addr(src.desc);
        if constexpr (SHARED_MAP) keys_sa = smem_addr(src.keys);
    }
    // plan of the first tour: largest p with plan_tour_off[p] <= t
    int plan = warp_find_plan(a, c_begin * 32, lane);
    for (int c = c_begin; c < c_end; ++c) {
        const int t = c * 32 + lane;
        const bool active = t < a.n_tours;
        while (plan + 1 < a.n_plans && a.plan_tour_off[plan + 1] <= t) ++plan;
        if constexpr (!SHARED_MAP) src.map = a.slot_map + (int64_t)plan * a.slot_stride;
        // one pass over the tour's orders: check them, count the lines and
        // stage the first SHORT_MAX keys in this thread's buffer column.
        // Position p of the column is element (p >> 1) * 2T + (p & 1) (two
        // keys per slot, slots T apart): the write address wa advances by
        // stepb, which alternates between 1 and 2T - 1 elements, and by 2T
        // elements over two positions, so no position is recomputed per line.
        using KeyT = typename std::conditional<KEY16, uint16_t, uint32_t>::type;
        constexpr uint32_t KB = sizeof(KeyT);
        uint32_t wa = smem_addr(KEY16 ? static_cast<void*>(col16) : static_cast<void*>(col32));
        const uint32_t two_tb = 2u * (uint32_t)T * KB;
        uint32_t stepb = KB;
        int n = 0;
        bool bad = false;
        if (active) {
            const int q0 = __ldg(a.tour_off + t), q1 = __ldg(a.tour_off + t + 1);
            if (q0 < 0 || q1 < q0 || (int64_t)q1 > a.n_seq) {
                flag(a.status, WH_STATUS_BAD_OFFSET);
                bad = true;
            } else if constexpr (SMEM_TABLES && SHARED_MAP) {
                // staged order book, shared slotting.  Software-pipelined:
                // order ids two ahead, descriptors one ahead.  A descriptor
                // is read at a clamped (always valid) index; an invalid id
                // reads as count 255, so one test per order catches invalid
                // ids, orders the short path does not take and tours over
                // SHORT_MAX lines, and only its exit tells them apart.
                const uint32_t o_max = (uint32_t)max(a.n_orders - 1, 0);
                auto desc_of = [&](int o) {
                    const uint32_t dv = lds_key<uint32_t>(desc_sa + 4u * min((uint32_t)o, o_max));
                    return (uint32_t)o < (uint32_t)a.n_orders ? dv : 0xFFFFFFFFu;
                };
                int o_a = q0 < q1 ? order_id<ID16>(a, q0) : 0;
                int o_b = q0 + 1 < q1 ? order_id<ID16>(a, q0 + 1) : 0;
                uint32_t d = desc_of(o_a);
                for (int q = q0; q < q1; ++q) {
                    const int o = o_a;
                    o_a = o_b;
                    const uint32_t dn = desc_of(o_a);
                    o_b = q + 2 < q1 ? order_id<ID16>(a, q + 2) : 0;
                    const int c = (int)(d & 0xFFu);
                    if (n + c > SHORT_MAX) {
                        if ((uint32_t)o >= (uint32_t)a.n_orders) {
                            flag(a.status, WH_STATUS_BAD_ORDER);
                            bad = true;
                        } else {
                            n += c;   // the long-tour kernel takes (and checks) it
                        }
                        break;
                    }
                    n += c;
                    // two lines a step (positions p and p + 1 sit stepb bytes
                    // apart), then the odd one, predicated
                    uint32_t sa = keys_sa + (d >> 8) * KB;
                    const uint32_t se = sa + (uint32_t)c * KB;
                    for (; sa + KB < se; sa += 2 * KB) {
                        const uint32_t k0 = lds_key<KeyT>(sa), k1 = lds_key<KeyT>(sa + KB);
                        sts_key<KeyT>(wa, k0);
                        sts_key<KeyT>(wa + stepb, k1);
                        wa += two_tb;
                    }
                    const bool odd = sa < se;
                    sts_key_if<KeyT>(odd, wa, lds_key_if<KeyT>(odd, sa));
                    wa += odd ? stepb : 0u;
                    stepb = odd ? two_tb - stepb : stepb;
                    d = dn;
                }
            } else {
                // software-pipelined: order ids two ahead, descriptors one ahead
                int o2 = q0 + 1 < q1 ? order_id<ID16>(a, q0 + 1) : 0;
                uint32_t d1 = 0;
                int o1 = 0;
                if (q0 < q1) {
                    o1 = order_id<ID16>(a, q0);
                    if constexpr (SMEM_TABLES)
                        d1 = (unsigned)o1 < (unsigned)a.n_orders ? lds_key<uint32_t>(desc_sa + 4u * (uint32_t)o1) : 0xFFFFFFFFu;
                }
                for (int q = q0; q < q1; ++q) {
                    const int o = o1;
                    const uint32_t d = d1;
                    o1 = o2;
                    if constexpr (SMEM_TABLES)
                        d1 = (q + 1 < q1 && (unsigned)o1 < (unsigned)a.n_orders) ? lds_key<uint32_t>(desc_sa + 4u * (uint32_t)o1)
                                                                                  : 0xFFFFFFFFu;
                    o2 = q + 2 < q1 ? order_id<ID16>(a, q + 2) : 0;
                    if ((unsigned)o >= (unsigned)a.n_orders) { flag(a.status, WH_STATUS_BAD_ORDER); bad = true; break; }
                    int lb, le;
                    if constexpr (SMEM_TABLES) {
                        lb = (int)(d >> 8);
                        le = lb + (int)(d & 0xFFu);
                        if ((d & 0xFFu) == 0xFFu) { n = SHORT_MAX + 1; break; }   // long-tour kernel checks it
                    } else {
                        lb = src.off[o];
                        le = src.off[o + 1];
                        if (lb < 0 || le < lb || le > a.n_lines) { flag(a.status, WH_STATUS_BAD_OFFSET); bad = true; break; }
                    }
                    if (n + (le - lb) > SHORT_MAX) { n += le - lb; break; }
                    n += le - lb;
                    if constexpr (!SHARED_MAP && !KEY16) {
                        // the plan's own slotting, 32-bit keys: the lines'
                        // SKUs go to their positions here; the pass after
                        // the order loop turns them into keys, eight
                        // slot-map gathers in flight whatever the orders' sizes
                        int l = lb;
                        for (; l + 1 < le; l += 2) {
                            const uint32_t s0 = (uint32_t)src.skus[l], s1 = (uint32_t)src.skus[l + 1];
                            sts_key<uint32_t>(wa, s0);
                            sts_key<uint32_t>(wa + stepb, s1);
                            wa += two_tb;
                        }
                        if (l < le) {
                            sts_key<uint32_t>(wa, (uint32_t)src.skus[l]);
                            wa += stepb;
                            stepb = two_tb - stepb;
                        }
                        continue;
                    } else if constexpr (!SHARED_MAP) {
                        // the plan's own slotting: four lines a step, their
                        // SKUs and then their slot-map gathers (global
                        // memory) in flight together
                        for (int l0 = lb; l0 < le; l0 += 4) {
                            int sk[4], loc[4];
#pragma unroll
                            for (int j = 0; j < 4; ++j) sk[j] = l0 + j < le ? src.skus[l0 + j] : 0;
#pragma unroll
                            for (int j = 0; j < 4; ++j)
                                loc[j] = (l0 + j < le && (unsigned)sk[j] < (unsigned)a.n_sku) ? src.map[sk[j]] : -1;
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                if (l0 + j >= le) continue;
                                uint32_t k32 = KEY_BAD;
                                if ((unsigned)sk[j] >= (unsigned)a.n_sku) flag(a.status, WH_STATUS_BAD_SKU);
                                else if ((unsigned)loc[j] >= (unsigned)a.g.n_loc) flag(a.status, WH_STATUS_BAD_LOC);
                                else k32 = loc_key(a.g, loc[j]);
                                sts_key<KeyT>(wa, KEY16 ? key16_of(k32) : k32);
                                wa += stepb;
                                stepb = two_tb - stepb;
                            }
                        }
                        continue;
                    }
                    // two lines a step (positions p and p + 1 sit `stepb`
                    // bytes apart), then the odd one
                    if constexpr (SMEM_TABLES) {
                        uint32_t sa = keys_sa + (uint32_t)lb * KB;
                        const uint32_t se = keys_sa + (uint32_t)le * KB;
                        for (; sa + KB < se; sa += 2 * KB) {
                            const uint32_t k0 = lds_key<KeyT>(sa), k1 = lds_key<KeyT>(sa + KB);
                            sts_key<KeyT>(wa, k0);
                            sts_key<KeyT>(wa + stepb, k1);
                            wa += two_tb;
                        }
                        if (sa < se) {
                            sts_key<KeyT>(wa, lds_key<KeyT>(sa));
                            wa += stepb;
                            stepb = two_tb - stepb;
                        }
                    } else {
                        int l = lb;
                        for (; l + 1 < le; l += 2) {
                            const uint32_t k0 = key_of<KEY16, SHARED_MAP, SMEM_TABLES>(a, src, l);
                            const uint32_t k1 = key_of<KEY16, SHARED_MAP, SMEM_TABLES>(a, src, l + 1);
                            sts_key<KeyT>(wa, k0);
                            sts_key<KeyT>(wa + stepb, k1);
                            wa += two_tb;
                        }
                        if (l < le) {
                            sts_key<KeyT>(wa, key_of<KEY16, SHARED_MAP, SMEM_TABLES>(a, src, l));
                            wa += stepb;
                            stepb = two_tb - stepb;
                        }
                    }
                }
            }
        }
        if constexpr (!SHARED_MAP && !KEY16) {
            // positions 0 .. n-1 hold SKUs: their slots, eight at a time
            const int np = (active && !bad && n <= SHORT_MAX) ? n : 0;
            const uint32_t cb = smem_addr(col32);
            for (int p0 = 0; p0 < np; p0 += 8) {
                uint32_t sk[8];
                int loc[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int p = p0 + j;
                    sk[j] = p < np ? lds_key<uint32_t>(cb + (uint32_t)(p >> 1) * (8u * (uint32_t)T) + 4u * (uint32_t)(p & 1)) : 0u;
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) loc[j] = (p0 + j < np && sk[j] < (uint32_t)a.n_sku) ? src.map[sk[j]] : -1;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int p = p0 + j;
                    if (p >= np) continue;
                    uint32_t k32 = KEY_BAD;
                    if (sk[j] >= (uint32_t)a.n_sku) flag(a.status, WH_STATUS_BAD_SKU);
                    else if ((unsigned)loc[j] >= (unsigned)a.g.n_loc) flag(a.status, WH_STATUS_BAD_LOC);
                    else k32 = loc_key(a.g, loc[j]);
                    sts_key<uint32_t>(cb + (uint32_t)(p >> 1) * (8u * (uint32_t)T) + 4u * (uint32_t)(p & 1), k32);
                }
            }
        }
        bool is_long = active && !bad && n > SHORT_MAX;
        if (is_long && !defer_long(a, inst, t, plan)) { is_long = false; bad = true; }
        const bool run = active && !bad && !is_long;
        const int nr = run ? n : 0;
        const int nmax = __reduce_max_sync(0xffffffffu, nr);
        int cs = 0, cr = 0, m = 0;
        bool kbad = false;   // a line whose SKU or slot is invalid (its key is the bad-key marker)
        if constexpr (KEY16) {
            if (nmax <= 16) tour16<8>(a, col16, T, nr, need_rr, cs, cr, m, check_keys, &kbad);
            else if (nmax <= 32) tour16<16>(a, col16, T, nr, need_rr, cs, cr, m, check_keys, &kbad);
            else tour16<32>(a, col16, T, nr, need_rr, cs, cr, m, check_keys, &kbad);
        } else {
            if (nmax <= 16) tour32<16>(a, col32, T, nr, need_rr, cs, cr, m, check_keys, &kbad);
            else if (nmax <= 32) tour32<32>(a, col32, T, nr, need_rr, cs, cr, m, check_keys, &kbad);
            else tour32<64>(a, col32, T, nr, need_rr, cs, cr, m, check_keys, &kbad);
        }
        kbad = kbad && run;
        // more pick aisles than this thread's record slots: the long-tour
        // pass scores the tour
        bool rec_long = run && !kbad && need_rr && m > a.max_rec;
        if (rec_long && !defer_long(a, inst, t, plan)) {
            rec_long = false;
            bad = true;
        }
        const bool ok = run && !kbad && !rec_long && !bad;
        if (active && (bad || kbad)) {
            if (a.tour_s) a.tour_s[t] = -1;
            if (a.tour_rr) a.tour_rr[t] = -1;
        } else if (ok) {
            if (a.tour_s && want_s) a.tour_s[t] = cs;
            if (a.tour_rr && need_rr) a.tour_rr[t] = cr;
        }
        const int key = active ? plan : -1;
        const long long ss = segmented_sum(ok ? cs : 0, key, lane);
        const long long sr = segmented_sum(ok ? cr : 0, key, lane);
        const int prev_key = __shfl_up_sync(0xffffffffu, key, 1);
        if (active && (lane == 0 || prev_key != key)) {
            if (a.plan_s && want_s && ss) atomicAdd(reinterpret_cast<unsigned long long*>(&a.plan_s[plan]), (unsigned long long)ss);
            if (a.plan_rr && need_rr && sr) atomicAdd(reinterpret_cast<unsigned long long*>(&a.plan_rr[plan]), (unsigned long long)sr);
        }
    }
}

// Per-order aggregate for the S-shape rule on <= 64 aisles: the bitmask of
// the aisles its lines visit, its largest key (aisle << 16 | slot: the
// rightmost aisle and that aisle's deepest pick) and flags (1: a line with an
// invalid SKU or slot, 2: at least one valid line, 4: malformed offsets).
__device__ __forceinline__ uint4 order_aggregate(const EvalArgs& a, int o) {
    const int lb = a.order_off[o], le = a.order_off[o + 1];
    uint64_t bits = 0;
    uint32_t kmax = 0, fl = 0;
    if (lb < 0 || le < lb || le > a.n_lines) {
        flag(a.status, WH_STATUS_BAD_OFFSET);
        fl = 4u;
    } else {
        // four lines a step: their SKU loads, then their slot loads, in
        // flight together
        for (int l0 = lb; l0 < le; l0 += 4) {
            int sku[4], loc[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) sku[j] = l0 + j < le ? a.line_sku[l0 + j] : -1;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                loc[j] = -1;
                if (l0 + j >= le) continue;
                if ((unsigned)sku[j] >= (unsigned)a.n_sku) {
                    flag(a.status, WH_STATUS_BAD_SKU);
                    fl |= 1u;
                    continue;
                }
                loc[j] = a.slot_map[sku[j]];
                if ((unsigned)loc[j] >= (unsigned)a.g.n_loc) {
                    flag(a.status, WH_STATUS_BAD_LOC);
                    fl |= 1u;
                    loc[j] = -1;
                }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (loc[j] < 0) continue;
                const uint32_t key = loc_key(a.g, loc[j]);
                bits |= 1ull << (key >> 16);
                kmax = max(kmax, key);
                fl |= 2u;
            }
        }
    }
    return make_uint4((uint32_t)bits, (uint32_t)(bits >> 32), kmax, fl);
}

// line keys of one instance, zeroed plan sums, plan offset checks
__device__ __forceinline__ void prep_instance(const EvalArgs& a, uint32_t mask, int i0, int stride) {
    if (a.line_key) {
        uint32_t* line_key = const_cast<uint32_t*>(a.line_key);
        for (int l = i0; l < a.n_lines; l += stride) {
            const int sku = a.line_sku[l];
            uint32_t key = KEY_BAD;
            if ((unsigned)sku >= (unsigned)a.n_sku) {
                flag(a.status, WH_STATUS_BAD_SKU);
            } else {
                const int loc = a.slot_map[sku];
                if ((unsigned)loc >= (unsigned)a.g.n_loc) flag(a.status, WH_STATUS_BAD_LOC);
                else key = loc_key(a.g, loc);
            }
            line_key[l] = key;
        }
    }
    if (a.order_agg)
        for (int o = i0; o < a.n_orders; o += stride) a.order_agg[o] = order_aggregate(a, o);
    const bool zs = a.plan_s && (mask & WH_ROUTE_SSHAPE);
    const bool zr = a.plan_rr && (mask & WH_ROUTE_OPTIMAL);
    for (int p = i0; p < a.n_plans; p += stride) {
        if (zs) a.plan_s[p] = 0;
        if (zr) a.plan_rr[p] = 0;
        const int t0 = a.plan_tour_off[p], t1 = a.plan_tour_off[p + 1];
        if (t0 < 0 || t1 < t0 || t1 > a.n_tours || (p == 0 && t0 != 0) || (p == a.n_plans - 1 && t1 != a.n_tours))
            flag(a.status, WH_STATUS_BAD_OFFSET);
    }
}

// ------------------------------------------------------------------ kernels

__global__ void k_prep(EvalArgs a) {
    const int i0 = blockIdx.x * blockDim.x + threadIdx.x;   // (lines, orders and plans by grid stride)
    if (i0 == 0) *a.long_count = 0;
    prep_instance(a, a.mask, i0, gridDim.x * blockDim.x);
}

// one block row per instance (blockIdx.y); block (0,0) resets the counters
__global__ void k_prep_batch(BatchArgs b) {
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
        *b.queue = 0;
        *b.long_count = 0;
    }
    for (int i = blockIdx.y; i < b.n_inst; i += gridDim.y)
        prep_instance(b.insts[i], b.mask, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// 16-bit keys: 384-thread CTAs, two per SM (24 warps; 85 registers a thread
// fit the sort without spills, and one copy of the order book per CTA keeps
// the shared-memory tables at two copies per SM); 32-bit keys: 256 threads
template <bool KEY16, bool SHARED_MAP, bool SMEM_TABLES>
__global__ void __launch_bounds__(KEY16 ? 384 : 256, 2) k_eval_short(EvalArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31;
    uint32_t* s_desc = reinterpret_cast<uint32_t*>(smem);
    void* s_tab = smem + sizeof(uint32_t) * (size_t)a.n_orders;
    size_t off_b = 0;
    if (SMEM_TABLES)
        off_b = (sizeof(uint32_t) * (size_t)a.n_orders + (SHARED_MAP ? (KEY16 ? 2 : 4) : 4) * (size_t)a.n_lines + 15) &
                ~(size_t)15;
    unsigned char* buf_base = smem + off_b;

    KeySrc src = global_src(a);
    bool check_keys = true;   // keys read from global memory: every tour checks its own
    if constexpr (SMEM_TABLES) check_keys = __syncthreads_or(stage_tables<KEY16, SHARED_MAP>(a, s_desc, s_tab, src, tid, T));
    // this warp's contiguous range of 32-tour chunks
    int c_begin, c_end;
    warp_chunk_range(a, c_begin, c_end);
    if (c_begin >= c_end) return;
    eval_chunks<KEY16, SHARED_MAP, SMEM_TABLES>(a, src, a.mask, 0, c_begin, c_end,
                                                reinterpret_cast<uint32_t*>(buf_base) + tid,
                                                reinterpret_cast<uint2*>(buf_base) + tid, T, lane, check_keys);
}

// S-shape only (routing mask = S-shape): no sort.  The S-shape length of a
// tour depends only on its number of pick aisles, its rightmost pick aisle
// and that aisle's deepest pick (the closed form of Eq. (2) under the S-shape
// rule), so one pass over the lines marks the visited aisles in a per-thread
// shared-memory bitmap and keeps the rightmost aisle's deepest slot.  Tours of
// any length stay in their thread (nothing is deferred); few registers, so
// many warps hide the gather latency.
constexpr int SSHAPE_MAX_WORDS = 64;   // bitmap words per thread: A <= 2048

template <bool KEY16, bool SHARED_MAP, bool SMEM_TABLES>
__global__ void __launch_bounds__(256) k_eval_sshape(EvalArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31;
    uint32_t* s_desc = reinterpret_cast<uint32_t*>(smem);
    void* s_tab = smem + sizeof(uint32_t) * (size_t)a.n_orders;
    size_t off_b = 0;
    if (SMEM_TABLES)
        off_b = (sizeof(uint32_t) * (size_t)a.n_orders + (SHARED_MAP ? (KEY16 ? 2 : 4) : 4) * (size_t)a.n_lines + 15) &
                ~(size_t)15;
    uint32_t* bm = reinterpret_cast<uint32_t*>(smem + off_b) + tid;   // word w at bm[w * T]
    const int nw = (a.g.A + 31) >> 5;
    KeySrc src = global_src(a);
    if constexpr (SMEM_TABLES) {
        stage_tables<KEY16, SHARED_MAP>(a, s_desc, s_tab, src, tid, T);   // the loop checks every key
        __syncthreads();
    }
    for (int w = 0; w < nw; ++w) bm[w * T] = 0u;
    int c_begin, c_end;
    warp_chunk_range(a, c_begin, c_end);
    if (c_begin >= c_end) return;
    int plan = warp_find_plan(a, c_begin * 32, lane);
    for (int c = c_begin; c < c_end; ++c) {
        const int t = c * 32 + lane;
        const bool active = t < a.n_tours;
        while (plan + 1 < a.n_plans && a.plan_tour_off[plan + 1] <= t) ++plan;
        if constexpr (!SHARED_MAP) src.map = a.slot_map + (int64_t)plan * a.slot_stride;
        int m = 0, r = -1, dr = 0;
        bool bad = false, kbad = false;
        if (active) {
            const int q0 = __ldg(a.tour_off + t), q1 = __ldg(a.tour_off + t + 1);
            if (q0 < 0 || q1 < q0 || (int64_t)q1 > a.n_seq) {
                flag(a.status, WH_STATUS_BAD_OFFSET);
                bad = true;
            } else {
                // one flat loop over the tour's lines (one line per lane per
                // iteration; a lane opens its next order when the current one
                // is used up), so lanes stay in step whatever the order sizes
                int q = q0, l = 0, le = 0;
                int o_next = q0 < q1 ? __ldg(a.order_seq + q0) : 0;
                for (;;) {
                    bool more = true;
                    while (l == le) {
                        if (q == q1) { more = false; break; }
                        const int o = o_next;
                        ++q;
                        o_next = q < q1 ? __ldg(a.order_seq + q) : 0;
                        if ((unsigned)o >= (unsigned)a.n_orders) {
                            flag(a.status, WH_STATUS_BAD_ORDER);
                            bad = true;
                            more = false;
                            break;
                        }
                        bool global = true;
                        if constexpr (SMEM_TABLES) {
                            const uint32_t d = src.desc[o];
                            if ((d & 0xFFu) != 0xFFu) {
                                l = (int)(d >> 8);
                                le = l + (int)(d & 0xFFu);
                                global = false;
                            }
                        }
                        if (global) {
                            l = src.off[o];
                            le = src.off[o + 1];
                            if (l < 0 || le < l || le > a.n_lines) {
                                flag(a.status, WH_STATUS_BAD_OFFSET);
                                bad = true;
                                more = false;
                                break;
                            }
                        }
                    }
                    if (!more) break;
                    const uint32_t key = key_of<KEY16, SHARED_MAP, SMEM_TABLES>(a, src, l);
                    ++l;
                    if (key == (KEY16 ? KEY16_BAD : KEY_BAD)) {
                        kbad = true;
                        continue;
                    }
                    const int ai = (int)(KEY16 ? key >> 8 : key >> 16);
                    const int dk = (int)(KEY16 ? key & 0xFFu : key & 0xFFFFu);
                    uint32_t* wp = bm + (ai >> 5) * T;
                    const uint32_t bit = 1u << (ai & 31), wv = *wp;
                    if (!(wv & bit)) {
                        *wp = wv | bit;
                        ++m;
                    }
                    dr = ai > r ? dk : (ai == r ? max(dr, dk) : dr);
                    r = max(r, ai);
                }
            }
            if (m > 0)
                for (int w = 0; w < nw; ++w) bm[w * T] = 0u;
        }
        const bool ok = active && !bad && !kbad;
        const int cs = ok ? sshape_cost(a.g, m, r, dr) : 0;
        if (active && !ok) {
            if (a.tour_s) a.tour_s[t] = -1;
        } else if (ok && a.tour_s) {
            a.tour_s[t] = cs;
        }
        const int key = active ? plan : -1;
        const long long ss = segmented_sum(cs, key, lane);
        const int prev_key = __shfl_up_sync(0xffffffffu, key, 1);
        if (active && (lane == 0 || prev_key != key) && a.plan_s && ss)
            atomicAdd(reinterpret_cast<unsigned long long*>(&a.plan_s[plan]), (unsigned long long)ss);
    }
}

constexpr int SSHAPE_AGG_THREADS = 256;

// S-shape only with per-order aggregates (shared slotting, <= 64 aisles):
// a tour's pick-aisle set is the union of its orders' aisle sets and its
// rightmost aisle's deepest pick is the largest key over its orders, so each
// tour merges one 16-byte record per order (no per-line work).  No shared
// memory: full occupancy hides the order-id and record loads.
// One warp's 32-tour chunks [c_begin, c_end): each tour merges the aggregates
// of its orders (agg(o) -> uint4), then the S-shape closed form and the
// segmented plan sums.
template <typename Agg>
__device__ __forceinline__ void sshape_agg_chunks(const EvalArgs& a, Agg agg, int c_begin, int c_end, int lane) {
    const bool vec = (reinterpret_cast<uintptr_t>(a.order_seq) & 15u) == 0;
    int plan = warp_find_plan(a, c_begin * 32, lane);
    for (int c = c_begin; c < c_end; ++c) {
        const int t = c * 32 + lane;
        const bool active = t < a.n_tours;
        while (plan + 1 < a.n_plans && a.plan_tour_off[plan + 1] <= t) ++plan;
        uint64_t bits = 0;
        uint32_t kmax = 0, fl = 0;
        bool bad = false;
        if (active) {
            const int q0 = __ldg(a.tour_off + t), q1 = __ldg(a.tour_off + t + 1);
            if (q0 < 0 || q1 < q0 || (int64_t)q1 > a.n_seq) {
                flag(a.status, WH_STATUS_BAD_OFFSET);
                bad = true;
            } else {
                auto take = [&](int o) {
                    if ((unsigned)o >= (unsigned)a.n_orders) {
                        bad = true;
                        return;
                    }
                    const uint4 r = agg(o);
                    bits |= (uint64_t)r.x | ((uint64_t)r.y << 32);
                    kmax = (r.w & 2u) ? max(kmax, r.z) : kmax;
                    fl |= r.w;
                };
                // the thread's run of order ids: scalar loads up to a 16-byte
                // boundary, then four ids per vector load (a quarter of the
                // load requests), then the tail
                int q = q0;
                if (vec) {
                    for (; q < q1 && (q & 3); ++q) take(__ldg(a.order_seq + q));
                    for (; q + 4 <= q1; q += 4) {
                        const int4 v = __ldg(reinterpret_cast<const int4*>(a.order_seq + q));
                        take(v.x);
                        take(v.y);
                        take(v.z);
                        take(v.w);
                    }
                }
                for (; q < q1; ++q) take(__ldg(a.order_seq + q));
                if (bad) flag(a.status, WH_STATUS_BAD_ORDER);
            }
        }
        const bool ok = active && !bad && !(fl & 5u);
        const int m = __popcll(bits);
        const int cs = ok ? sshape_cost(a.g, m, (int)(kmax >> 16), (int)(kmax & 0xFFFFu)) : 0;
        if (active && a.tour_s) a.tour_s[t] = ok ? cs : -1;
        const int key = active ? plan : -1;
        const long long ss = segmented_sum(cs, key, lane);
        const int prev_key = __shfl_up_sync(0xffffffffu, key, 1);
        if (active && (lane == 0 || prev_key != key) && a.plan_s && ss)
            atomicAdd(reinterpret_cast<unsigned long long*>(&a.plan_s[plan]), (unsigned long long)ss);
    }
}


__global__ void __launch_bounds__(SSHAPE_AGG_THREADS) k_eval_sshape_agg(EvalArgs a) {
    int c_begin, c_end;
    warp_chunk_range(a, c_begin, c_end);
    if (c_begin >= c_end) return;
    sshape_agg_chunks(a, [&](int o) { return __ldg(a.order_agg + o); }, c_begin, c_end, threadIdx.x & 31);
}

// Persistent batch kernel: CTAs pop work items (instance, chunk range) from
// a queue ordered largest first, stage that instance's order book once, and
// split the item's chunks among their warps.
// 16-bit keys: up to 384-thread CTAs, two per SM (85 registers a thread, as
// k_eval_short); 32-bit keys: up to 256 threads.  ID16: the instances' order
// ids are read as 16-bit values.
template <bool KEY16, bool SMEM_TABLES, bool ID16>
__global__ void __launch_bounds__(KEY16 ? 384 : 256, 2) k_eval_batch(BatchArgs b) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item;
    __shared__ __align__(16) EvalArgs s_a;
    const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = T >> 5;
    uint32_t* s_desc = reinterpret_cast<uint32_t*>(smem);
    void* s_tab = smem + sizeof(uint32_t) * (size_t)b.max_orders;
    size_t off_b = 0;
    if (SMEM_TABLES)
        off_b = (sizeof(uint32_t) * (size_t)b.max_orders + (KEY16 ? 2 : 4) * (size_t)b.max_lines + 15) & ~(size_t)15;
    unsigned char* buf_base = smem + off_b;
    uint32_t* col16 = reinterpret_cast<uint32_t*>(buf_base) + tid;
    uint2* col32 = reinterpret_cast<uint2*>(buf_base) + tid;
    int staged = -1;
    bool check_keys = true;   // the staged instance has a bad key (or keys are not staged)
    KeySrc src;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(b.queue, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= b.n_items) break;
        const WorkItem w = b.items[it];
        if (w.inst != staged) {
            const int* srcw = reinterpret_cast<const int*>(b.insts + w.inst);
            int* dstw = reinterpret_cast<int*>(&s_a);
            for (int i = tid; i < (int)(sizeof(EvalArgs) / sizeof(int)); i += T) dstw[i] = srcw[i];
            __syncthreads();
            src = global_src(s_a);
            bool kb = true;
            if constexpr (SMEM_TABLES) kb = stage_tables<KEY16, true>(s_a, s_desc, s_tab, src, tid, T);
            check_keys = kb;
            staged = w.inst;
        }
        check_keys = __syncthreads_or(check_keys);
        const int n = w.chunk_end - w.chunk_begin;
        const int cb = w.chunk_begin + warp * n / nw;   // the item's chunks split evenly over the warps
        const int ce = w.chunk_begin + (warp + 1) * n / nw;
        if (cb < ce)
            eval_chunks<KEY16, true, SMEM_TABLES, ID16>(s_a, src, b.mask, w.inst, cb, ce, col16, col32, T, lane,
                                                        check_keys);
        __syncthreads();
    }
}

// One warp per deferred tour (more than SHORT_MAX lines): keys gathered into
// a per-warp shared-memory buffer (lanes over orders, four lines' loads in
// flight), bitonic-sorted there.  With record scratch (L.rec): the per-aisle
// records are extracted in parallel (a ballot numbers the aisle runs) into
// the warp's slice, column j for the warp's j-th tour of a group of 32, and
// once the group is complete each lane runs the DP of one tour; a tour with
// more than LONG_RMAX records runs its scan and DP on one lane at once.
// Without scratch every tour's scan and DP run on one lane.
constexpr int LONG_RMAX = 48;   // records per tour kept for the per-lane DP

template <bool SHARED_MAP>
__global__ void __launch_bounds__(LONG_WARPS * 32, 6) k_eval_long(LongArgs L) {
    __shared__ uint32_t buf[LONG_WARPS][LONG_MAXL];
    __shared__ int s_meta[LONG_WARPS][32][4];   // inst, tour, plan, record count (-1: done)
    __shared__ uint32_t s_last[LONG_WARPS][32];  // largest key of the tour
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int count = min(*L.count, L.cap);
    uint32_t* kb = buf[warp];
    const bool need_rr = (L.mask & WH_ROUTE_OPTIMAL) != 0;
    const bool want_s = (L.mask & WH_ROUTE_SSHAPE) != 0;
    const int gw = blockIdx.x * LONG_WARPS + warp, n_warps = gridDim.x * LONG_WARPS;
    uint2* rec = L.rec ? L.rec + (int64_t)gw * LONG_RMAX * 32 : nullptr;   // [r][32]
    auto commit = [&](const EvalArgs& a, int t, int plan, int cs, int cr) {
        if (a.tour_s && want_s) a.tour_s[t] = cs;
        if (a.tour_rr && need_rr) a.tour_rr[t] = cr;
        if (a.plan_s && want_s) atomicAdd(reinterpret_cast<unsigned long long*>(&a.plan_s[plan]), (unsigned long long)cs);
        if (a.plan_rr && need_rr)
            atomicAdd(reinterpret_cast<unsigned long long*>(&a.plan_rr[plan]), (unsigned long long)cr);
    };
    // The warp's tours are gw, gw + n_warps, gw + 2 n_warps, ..., taken 32 at
    // a time.  Their headers are fetched ahead, so that the chain list entry
    // -> tour offsets -> order ids does not stall every tour: list entries
    // two tours ahead, offsets one tour ahead (at the start of a tour) and
    // the next tour's first 32 order ids once this tour's lines are gathered.
    auto list_of = [&](int w, int& inst, int& t, int& plan) {
        inst = L.list[3 * w];
        t = L.list[3 * w + 1];
        plan = L.list[3 * w + 2];
    };
    auto offs_of = [&](int inst, int t, int& q0, int& q1) {
        const int32_t* to = L.insts ? L.insts[inst].tour_off : L.single.tour_off;
        q0 = to[t];   // checked by the short kernel
        q1 = to[t + 1];
    };
    auto id_of = [&](int inst, int q) {
        const EvalArgs& a = L.insts ? L.insts[inst] : L.single;
        return a.order_seq16 ? (int)a.order_seq16[q] : a.order_seq[q];
    };
    int c_inst = 0, c_t = 0, c_plan = 0, c_q0 = 0, c_q1 = 0, c_o = 0;   // the next tour
    int n_inst = 0, n_t = 0, n_plan = 0;                                 // the one after
    if (gw < count) {
        list_of(gw, c_inst, c_t, c_plan);
        offs_of(c_inst, c_t, c_q0, c_q1);
        c_o = c_q0 + lane < c_q1 ? id_of(c_inst, c_q0 + lane) : 0;
    }
    if (gw + n_warps < count) list_of(gw + n_warps, n_inst, n_t, n_plan);
    for (int w0 = gw; w0 < count; w0 += 32 * n_warps) {
        int in_group = 0;
        for (int j = 0; j < 32; ++j) {
            const int w = w0 + j * n_warps;
            if (w >= count) break;
            in_group = j + 1;
            const int inst = c_inst, t = c_t, plan = c_plan, q0 = c_q0, q1 = c_q1, o_first = c_o;
            const bool more1 = w + n_warps < count;
            c_inst = n_inst;
            c_t = n_t;
            c_plan = n_plan;
            if (more1) offs_of(c_inst, c_t, c_q0, c_q1);
            if (w + 2 * n_warps < count) list_of(w + 2 * n_warps, n_inst, n_t, n_plan);
            const EvalArgs& a = L.insts ? L.insts[inst] : L.single;
            KeySrc src = global_src(a);
            if constexpr (!SHARED_MAP) src.map = a.slot_map + (int64_t)plan * a.slot_stride;
            int n = 0;
            bool bad = false;
            for (int qb = q0; qb < q1; qb += 32) {
                const int q = qb + lane;
                int lb = 0, le = 0;
                if (q < q1) {
                    // in range: checked by the short kernel
                    const int o = qb == q0 ? o_first : id_of(inst, q);
                    lb = a.order_off[o];
                    le = a.order_off[o + 1];
                    if (lb < 0 || le < lb || le > a.n_lines) {
                        flag(a.status, WH_STATUS_BAD_OFFSET);
                        bad = true;
                        lb = le = 0;
                    }
                }
                const int cnt = le - lb;
                const int incl = warp_inclusive_scan(cnt);
                // the lines' indices at their positions in the tour (shared
                // stores only); their keys are gathered below
                int pos = n + incl - cnt;
                for (int l = lb; l < le; ++l, ++pos)
                    if (pos < LONG_MAXL) kb[pos] = (uint32_t)l;
                n += __shfl_sync(0xffffffffu, incl, 31);
            }
            if (more1) c_o = c_q0 + lane < c_q1 ? id_of(c_inst, c_q0 + lane) : 0;
            __syncwarp();
            // keys: the warp's lanes over the tour's positions, four positions
            // a lane with their SKU and slot loads in flight together
            {
                const int nn = min(n, LONG_MAXL);
                for (int x0 = 0; x0 < nn; x0 += 128) {
                    uint32_t k[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int x = x0 + 32 * u + lane;
                        k[u] = x < nn ? key_of<false, SHARED_MAP, false>(a, src, (int)kb[x]) : 0u;
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int x = x0 + 32 * u + lane;
                        if (x < nn) {
                            bad |= (k[u] == KEY_BAD);
                            kb[x] = k[u];
                        }
                    }
                }
            }
            bad = __any_sync(0xffffffffu, bad);
            if (n > LONG_MAXL || bad) {
                if (lane == 0) {
                    if (n > LONG_MAXL) flag(a.status, WH_STATUS_TOUR_TOO_LONG);
                    if (a.tour_s) a.tour_s[t] = -1;
                    if (a.tour_rr) a.tour_rr[t] = -1;
                    s_meta[warp][j][3] = -1;
                }
                __syncwarp();
                continue;
            }
            warp_sort_buffer(kb, n, lane);
            int m = 0;
            if (rec) {
                // per-aisle records: run r of the sorted keys -> rec[r][j]
                for (int x0 = 0; x0 < n; x0 += 32) {
                    const int x = x0 + lane;
                    const bool in = x < n;
                    const uint32_t key = in ? kb[x] : 0u;
                    const int ai = (int)(key >> 16);
                    const bool first = in && (x == 0 || (int)(kb[x - 1] >> 16) != ai);
                    const bool last = in && (x == n - 1 || (int)(kb[x + 1] >> 16) != ai);
                    const unsigned fm = __ballot_sync(0xffffffffu, first);
                    const int r = m + __popc(fm & ((2u << lane) - 1u)) - 1;
                    if (last && r < LONG_RMAX) {
                        const int hi = (int)(key & 0xFFFFu);
                        int lo = hi, gi = 0;
                        for (int y = x; y > 0 && (int)(kb[y - 1] >> 16) == ai; --y) {
                            const int kp = (int)(kb[y - 1] & 0xFFFFu);
                            gi = max(gi, lo - kp);
                            lo = kp;
                        }
                        rec[r * 32 + j] = make_uint2(((uint32_t)ai << 16) | (uint32_t)lo, ((uint32_t)hi << 16) | (uint32_t)gi);
                    }
                    m += __popc(fm);
                }
            }
            if (lane == 0) {
                const uint32_t kl = kb[n - 1];   // rightmost aisle, its deepest slot
                if (rec && m <= LONG_RMAX) {
                    s_meta[warp][j][0] = inst;
                    s_meta[warp][j][1] = t;
                    s_meta[warp][j][2] = plan;
                    s_meta[warp][j][3] = m;
                    s_last[warp][j] = kl;
                } else {
                    // the scan and the DP on this lane
                    DP5 v;
                    dp_init(v);
                    int mm = 0, pa = 0, lo = 0, prev = 0, gi = 0;
                    for (int i = 0; i < n; ++i) {
                        const uint32_t key = kb[i];
                        const int ai = (int)(key >> 16), k = (int)(key & 0xFFFFu);
                        const bool first = (i == 0) || ((int)(kb[i - 1] >> 16) != ai);
                        const bool last = (i == n - 1) || ((int)(kb[i + 1] >> 16) != ai);
                        gi = first ? 0 : max(gi, k - prev);
                        lo = first ? k : lo;
                        prev = k;
                        if (last) {
                            if (need_rr) dp_aisle(v, a.g, ai - pa, lo, k, gi);
                            pa = ai;
                            ++mm;
                        }
                    }
                    commit(a, t, plan, sshape_cost(a.g, mm, (int)(kl >> 16), (int)(kl & 0xFFFFu)),
                           need_rr ? dp_final(v) : 0);
                    s_meta[warp][j][3] = -1;
                }
            }
            __syncwarp();
        }
        // the group's DPs, one tour per lane
        if (rec && lane < in_group) {
            const int m = s_meta[warp][lane][3];
            if (m >= 0) {
                const int inst = s_meta[warp][lane][0], t = s_meta[warp][lane][1], plan = s_meta[warp][lane][2];
                const EvalArgs& a = L.insts ? L.insts[inst] : L.single;
                const uint32_t kl = s_last[warp][lane];
                const int cr = need_rr ? rr_records32_mem(a.g, rec + lane, 32, m) : 0;
                commit(a, t, plan, sshape_cost(a.g, m, (int)(kl >> 16), (int)(kl & 0xFFFFu)), cr);
            }
        }
        __syncwarp();
    }
}

template <typename K>
cudaError_t grid_for(K kern, int threads, size_t smem, int num_sms, int want, int* grid) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int g = per_sm * num_sms;
    if (g > want) g = want;
    if (g < 1) g = 1;
    *grid = g;
    return cudaSuccess;
}

template <bool K16, bool SH, bool SM>
cudaError_t launch_short_t(const EvalArgs& a, const Tuning& t, size_t smem, int num_sms, cudaStream_t s,
                           int* grid_out) {
    auto kern = k_eval_short<K16, SH, SM>;
    const int warps_needed = (a.n_tours + 31) / 32;
    int grid = 0;
    cudaError_t e = grid_for(kern, t.threads, smem, num_sms, (warps_needed + t.threads / 32 - 1) / (t.threads / 32), &grid);
    if (e != cudaSuccess) return e;
    if (grid_out) *grid_out = grid;
    kern<<<grid, t.threads, smem, s>>>(a);
    return cudaGetLastError();
}

template <bool K16, bool SH, bool SM>
cudaError_t launch_sshape_t(const EvalArgs& a, const Tuning& t, size_t smem, int num_sms, cudaStream_t s,
                            int* grid_out) {
    auto kern = k_eval_sshape<K16, SH, SM>;
    const int warps_needed = (a.n_tours + 31) / 32;
    int grid = 0;
    cudaError_t e = grid_for(kern, t.threads, smem, num_sms, (warps_needed + t.threads / 32 - 1) / (t.threads / 32), &grid);
    if (e != cudaSuccess) return e;
    if (grid_out) *grid_out = grid;
    kern<<<grid, t.threads, smem, s>>>(a);
    return cudaGetLastError();
}

template <bool K16, bool SM, bool ID16>
cudaError_t launch_batch_t(const BatchArgs& b, const Tuning& t, size_t smem, int num_sms, cudaStream_t s) {
    auto kern = k_eval_batch<K16, SM, ID16>;
    int grid = 0;
    cudaError_t e = grid_for(kern, t.threads, smem, num_sms, b.n_items, &grid);
    if (e != cudaSuccess) return e;
    kern<<<grid, t.threads, smem, s>>>(b);
    return cudaGetLastError();
}

}  // namespace

bool key16_ok(const Geo& g) { return g.A <= 255 && g.L <= 256; }

bool sshape_kernel_applies(const EvalArgs& a) {
    return a.mask == WH_ROUTE_SSHAPE && (a.g.A + 31) / 32 <= SSHAPE_MAX_WORDS;
}


static size_t buffer_bytes(bool k16, int max_rec, int threads) {
    // a slot holds two keys or one record: 32 slots for 64 keys
    const size_t slots = max_rec > SHORT_MAX / 2 ? (size_t)max_rec : (size_t)(SHORT_MAX / 2);
    return (k16 ? sizeof(uint32_t) : sizeof(uint2)) * slots * (size_t)threads;
}

static size_t table_bytes(bool k16, bool shared_map, int64_t n_orders, int64_t n_lines) {
    const size_t b = sizeof(uint32_t) * (size_t)n_orders + (shared_map ? (k16 ? 2 : 4) : 4) * (size_t)n_lines;
    return (b + 15) & ~(size_t)15;
}

size_t eval_short_smem_bytes(const EvalArgs& a, const Tuning& t) {
    const bool k16 = t.key16 && key16_ok(a.g);
    size_t b = t.smem_tables ? table_bytes(k16, a.slot_stride == 0, a.n_orders, a.n_lines) : 0;
    return b + buffer_bytes(k16, a.max_rec, t.threads);
}

size_t eval_batch_smem_bytes(const BatchArgs& b, const Tuning& t, bool k16) {
    size_t s = t.smem_tables ? table_bytes(k16, true, b.max_orders, b.max_lines) : 0;
    return s + buffer_bytes(k16, b.max_rec, t.threads);
}

static cudaError_t launch_sshape(const EvalArgs& a, const Tuning& t, int num_sms, cudaStream_t s, int* grid_out) {
    if (a.order_agg) {
        int grid = 0;
        const int warps_needed = (a.n_tours + 31) / 32;
        const int want = (warps_needed + SSHAPE_AGG_THREADS / 32 - 1) / (SSHAPE_AGG_THREADS / 32);
        cudaError_t e = grid_for(k_eval_sshape_agg, SSHAPE_AGG_THREADS, 0, num_sms, want, &grid);
        if (e != cudaSuccess) return e;
        if (grid_out) *grid_out = grid;
        k_eval_sshape_agg<<<grid, SSHAPE_AGG_THREADS, 0, s>>>(a);
        return cudaGetLastError();
    }
    const bool shared_map = a.slot_stride == 0;
    const bool k16 = t.key16 && key16_ok(a.g);
    const bool sm = t.smem_tables != 0;
    const size_t smem = (sm ? table_bytes(k16, shared_map, a.n_orders, a.n_lines) : 0) +
                        sizeof(uint32_t) * (size_t)((a.g.A + 31) / 32) * (size_t)t.threads;
#define WH_LAUNCH(K, H, M) launch_sshape_t<K, H, M>(a, t, smem, num_sms, s, grid_out)
    if (k16) {
        if (shared_map) return sm ? WH_LAUNCH(true, true, true) : WH_LAUNCH(true, true, false);
        return sm ? WH_LAUNCH(true, false, true) : WH_LAUNCH(true, false, false);
    }
    if (shared_map) return sm ? WH_LAUNCH(false, true, true) : WH_LAUNCH(false, true, false);
    return sm ? WH_LAUNCH(false, false, true) : WH_LAUNCH(false, false, false);
#undef WH_LAUNCH
}

cudaError_t launch_prep(const EvalArgs& a, cudaStream_t s) {
    int work = a.n_plans;
    if (a.line_key && a.n_lines > work) work = a.n_lines;
    if (a.order_agg && a.n_orders > work) work = a.n_orders;
    int grid = (work + 255) / 256;
    if (grid > 4096) grid = 4096;
    if (grid < 1) grid = 1;
    k_prep<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_prep_batch(const BatchArgs& b, int max_work, cudaStream_t s) {
    int gx = (max_work + 255) / 256;
    if (gx > 16) gx = 16;
    if (gx < 1) gx = 1;
    const int gy = b.n_inst < 65535 ? b.n_inst : 65535;
    k_prep_batch<<<dim3(gx, gy), 256, 0, s>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_eval_short(const EvalArgs& a, const Tuning& tune, int num_sms, cudaStream_t s, int* grid_out) {
    const bool k16_ok = tune.key16 && key16_ok(a.g);
    if (tune.threads % 32 != 0 || tune.threads > (k16_ok ? 384 : 256) || tune.threads < 32) return cudaErrorInvalidValue;
    if (a.n_tours == 0) return cudaSuccess;
    if (sshape_kernel_applies(a)) {
        Tuning ts = tune;
        if (ts.threads > 256) ts.threads = 256;
        return launch_sshape(a, ts, num_sms, s, grid_out);
    }
    const Tuning& t = tune;
    const size_t smem = eval_short_smem_bytes(a, t);
    const bool shared_map = a.slot_stride == 0;
    const bool k16 = t.key16 && key16_ok(a.g);
    const bool sm = t.smem_tables != 0;
#define WH_LAUNCH(K, H, M) launch_short_t<K, H, M>(a, t, smem, num_sms, s, grid_out)
    if (k16) {
        if (shared_map) return sm ? WH_LAUNCH(true, true, true) : WH_LAUNCH(true, true, false);
        return sm ? WH_LAUNCH(true, false, true) : WH_LAUNCH(true, false, false);
    }
    if (shared_map) return sm ? WH_LAUNCH(false, true, true) : WH_LAUNCH(false, true, false);
    return sm ? WH_LAUNCH(false, false, true) : WH_LAUNCH(false, false, false);
#undef WH_LAUNCH
}

cudaError_t launch_eval_batch(const BatchArgs& b, const Tuning& t, bool k16, int num_sms, cudaStream_t s) {
    if (t.threads % 32 != 0 || t.threads > (k16 ? 384 : 256) || t.threads < 32) return cudaErrorInvalidValue;
    if (b.n_items == 0) return cudaSuccess;
    const size_t smem = eval_batch_smem_bytes(b, t, k16);
    const bool sm = t.smem_tables != 0;
#define WH_LAUNCH(K, M, I) launch_batch_t<K, M, I>(b, t, smem, num_sms, s)
    if (b.id16) {
        if (k16) return sm ? WH_LAUNCH(true, true, true) : WH_LAUNCH(true, false, true);
        return sm ? WH_LAUNCH(false, true, true) : WH_LAUNCH(false, false, true);
    }
    if (k16) return sm ? WH_LAUNCH(true, true, false) : WH_LAUNCH(true, false, false);
    return sm ? WH_LAUNCH(false, true, false) : WH_LAUNCH(false, false, false);
#undef WH_LAUNCH
}

// CTAs per SM of the long-tour kernel, the larger of its two forms: its grid
// (and its record scratch) is sized by this
static int long_per_sm() {
    int a = 0, b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_eval_long<true>, LONG_WARPS * 32, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_eval_long<false>, LONG_WARPS * 32, 0) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    const int m = a > b ? a : b;
    return m > 0 ? m : 1;
}

size_t long_rec_bytes(int num_sms) {
    const int per_sm = long_per_sm();
    if (per_sm < 1) return 0;
    return sizeof(uint2) * (size_t)LONG_RMAX * 32 * LONG_WARPS * (size_t)per_sm * (size_t)num_sms;
}

cudaError_t launch_eval_long(const LongArgs& L, bool shared_map, int num_sms, cudaStream_t s) {
    auto kern = shared_map ? k_eval_long<true> : k_eval_long<false>;
    const int per_sm = long_per_sm();
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    kern<<<num_sms * per_sm, LONG_WARPS * 32, 0, s>>>(L);
    return cudaGetLastError();
}


// 16-bit order ids (as shipped from the host when n_orders <= 65,536)
// widened to the int32 ids the evaluator reads: eight ids per thread step
// when both buffers are 16-byte aligned, one otherwise
namespace {
__global__ void k_widen_u16(const uint16_t* __restrict__ src, int32_t* __restrict__ dst, int64_t n, bool vec) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t done = 0;
    if (vec) {
        const int64_t n8 = n >> 3;
        const uint4* s8 = reinterpret_cast<const uint4*>(src);
        int4* d4 = reinterpret_cast<int4*>(dst);
        for (int64_t j = i; j < n8; j += stride) {
            const uint4 v = s8[j];
            d4[2 * j] = make_int4((int)(v.x & 0xFFFFu), (int)(v.x >> 16), (int)(v.y & 0xFFFFu), (int)(v.y >> 16));
            d4[2 * j + 1] = make_int4((int)(v.z & 0xFFFFu), (int)(v.z >> 16), (int)(v.w & 0xFFFFu), (int)(v.w >> 16));
        }
        done = n8 << 3;
    }
    for (int64_t j = done + i; j < n; j += stride) dst[j] = (int32_t)src[j];
}
}  // namespace

cudaError_t launch_widen_u16(const uint16_t* src, int32_t* dst, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const bool vec = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0;
    const int64_t work = vec ? (n >> 3) + 1 : n;
    int64_t grid = (work + 255) / 256;
    if (grid > 2048) grid = 2048;
    k_widen_u16<<<(int)grid, 256, 0, s>>>(src, dst, n, vec);
    return cudaGetLastError();
}

}  // namespace wh
