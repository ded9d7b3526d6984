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
#include "wh_internal.h"

namespace wh {

namespace {

constexpr int INF = 1 << 29;
constexpr uint32_t KEY_BAD = 0xFFFFFFFEu;   // a line whose SKU or slot is invalid
constexpr uint32_t KEY16_NONE = 0xFFFFu;
constexpr uint32_t KEY16_BAD = 0xFFFEu;
constexpr int LONG_WARPS = 4;
constexpr int LONG_MAXL = WH_MAX_TOUR_LINES;

__device__ __forceinline__ void flag(uint32_t* status, uint32_t bit) { atomicOr(status, bit); }

__device__ __forceinline__ uint32_t loc_key(const Geo& g, int loc) {
    const int two_l = 2 * g.L;
    const int a = loc / two_l;
    const int r = loc - a * two_l;          // side*L + k
    const int k = r >= g.L ? r - g.L : r;
    return ((uint32_t)a << 16) | (uint32_t)k;
}

// 32-bit key -> 16-bit key (aisle<<8 | slot); valid when A <= 255, L <= 256
__device__ __forceinline__ uint32_t key16_of(uint32_t k32) {
    if (k32 == KEY_BAD) return KEY16_BAD;
    return ((k32 >> 8) & 0xFF00u) | (k32 & 0xFFu);
}

// ---------------------------------------------------------------- DP state
// Five classes of a partial tour subgraph after an aisle, named by the degree
// of the aisle's front end a_j and back end b_j (0: not in the subgraph, E:
// even, U: odd) and the number of components: UU = (U,U,1C), E0 = (E,0,1C),
// OE = (0,E,1C), EE = (E,E,1C), E2 = (E,E,2C).
struct DP5 {
    int uu, e0, oe, ee, e2;
};

__device__ __forceinline__ void dp_init(DP5& v) {
    v.uu = INF; v.e0 = 0; v.oe = INF; v.ee = INF; v.e2 = INF;
}

// One aisle holding picks, reached d >= 0 aisles to the right of the previous
// one.  lo / hi: slot index of its shallowest / deepest pick; gi: largest gap
// between consecutive picks in slot units.
//
// No value is clamped at INF: every state value is min over partial tours of
// (start value 0 or INF) + that partial tour's length, and a partial tour is
// at most 4*x_{A-1} (horizontal) + 2*A*Y (vertical) < 2^28 by the layout
// bound 2*x_{A-1} + A*Y < 2^27, so values stay below INF + 2^28 + 2^28 = 2^30.
// __viaddmin_s32(a, b, c) = min(a + b, c) and __vimin3_s32 are the fused
// min-plus forms of those steps.
__device__ __forceinline__ void dp_aisle(DP5& v, const Geo& g, int d, int lo, int hi, int gi) {
    // cross the d aisle gaps: (1,1) for UU; (2,0) / (0,2) for E0 / OE, which
    // EE may also switch to; (2,2) for EE and E2
    const int h2 = 2 * g.P * d, h4 = h2 + h2;
    const int huu = v.uu + h2;
    const int he0 = min(v.e0, v.ee) + h2;
    const int hoe = min(v.oe, v.ee) + h2;
    const int hee = v.ee + h4;
    const int he2 = v.e2 + h4;
    // vertical options of this aisle: traverse Y, double traverse 2Y, leave
    // out the largest gap 2(Y-g), from the back 2(Y-y_lo), from the front 2*y_hi
    const int ylo = g.h + lo * g.S, yhi = g.h + hi * g.S;
    const int gap = __vimax3_s32(ylo, gi * g.S, g.Y - yhi);
    const int cG = 2 * (g.Y - gap), cB = 2 * (g.Y - ylo), cF = 2 * yhi;
    const int cT = g.Y, cD = 2 * g.Y;
    const int m3 = __vimin3_s32(he0, hoe, he2);
    v.uu = __viaddmin_s32(huu, cG, min(m3, hee) + cT);
    v.ee = __viaddmin_s32(huu, cT, __viaddmin_s32(m3, cD, hee + cG));
    v.e0 = he0 + cF;
    v.oe = hoe + cB;
    v.e2 = m3 + cG;
}

__device__ __forceinline__ int dp_final(const DP5& v) { return min(min(v.ee, v.e0), v.oe); }

// S-shape closed form from the number of pick aisles m, the rightmost pick
// aisle and its deepest slot.
__device__ __forceinline__ int sshape_cost(const Geo& g, int m, int last_a, int last_hi) {
    if (m == 0) return 0;
    const int d_r = g.h + last_hi * g.S;
    return 2 * last_a * g.P + ((m & 1) ? (m - 1) * g.Y + 2 * d_r : m * g.Y);
}

// ------------------------------------------------------ 32-bit key network
template <int N>
__device__ __forceinline__ void bitonic_sort(uint32_t (&x)[N]) {
#pragma unroll
    for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
            for (int i = 0; i < N; ++i) {
                const int l = i ^ j;
                if (l > i) {
                    const uint32_t a = x[i], b = x[l];
                    const uint32_t lo = min(a, b), hi = max(a, b);
                    if ((i & k) == 0) { x[i] = lo; x[l] = hi; }
                    else { x[i] = hi; x[l] = lo; }
                }
            }
        }
    }
}

// ------------------------------------------------------ 16-bit key network
// 2R positions in R registers: position p lives in register p % R, in the low
// half when p < R and the high half otherwise.  All-ascending bitonic sorter:
// each merge of block size k starts by comparing p with p ^ (k-1) (the
// mirrored partner), then half-cleans with p ^ j for j = k/4 .. 1.  For
// k <= R both halves run the same register pairs, so one 16x2 min/max pair
// serves two comparators; the final mirror step pairs halves across
// registers and needs a half swap.
template <int R>
__device__ __forceinline__ void sort16x2(uint32_t (&x)[R]) {
    constexpr int N = 2 * R;
#pragma unroll
    for (int k = 2; k <= N; k <<= 1) {
        if (k == N) {
#pragma unroll
            for (int r = 0; r < R / 2; ++r) {
                const uint32_t A = x[r], B = x[R - 1 - r];
                const uint32_t Bs = __byte_perm(B, 0, 0x1032);
                const uint32_t mn = __vminu2(A, Bs), mx = __vmaxu2(A, Bs);
                x[r] = __byte_perm(mn, mx, 0x7610);
                x[R - 1 - r] = __byte_perm(mn, mx, 0x5432);
            }
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int l = r ^ (k - 1);
                if (l > r) {
                    const uint32_t a = x[r], b = x[l];
                    x[r] = __vminu2(a, b);
                    x[l] = __vmaxu2(a, b);
                }
            }
        }
#pragma unroll
        for (int j = k >> 2; j > 0; j >>= 1) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int l = r ^ j;
                if (l > r) {
                    const uint32_t a = x[r], b = x[l];
                    x[r] = __vminu2(a, b);
                    x[l] = __vmaxu2(a, b);
                }
            }
        }
    }
}

// --------------------------------------------------------- record scans
// Sorted keys -> per-aisle records (rec[j*stride], at most cap of them) and
// the S-shape inputs (pick-aisle count, rightmost aisle, its deepest slot).
template <int N>
__device__ __forceinline__ void scan32(const uint32_t (&x)[N], uint2* rec, int stride, int cap, bool write,
                                       int& m, int& last_a, int& last_hi) {
    int lo = 0, prev = 0, gi = 0;
    m = 0; last_a = 0; last_hi = 0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const uint32_t key = x[i];
        const uint32_t a = key >> 16;
        const int k = (int)(key & 0xFFFFu);
        const bool first = (i == 0) || ((x[i - 1] >> 16) != a);
        const bool last = (i == N - 1) || ((x[i + 1] >> 16) != a);
        gi = first ? 0 : max(gi, k - prev);
        lo = first ? k : lo;
        prev = k;
        if (key != KEY_NONE && last) {
            if (write && m < cap) rec[m * stride] = make_uint2((a << 16) | (uint32_t)lo, ((uint32_t)k << 16) | (uint32_t)gi);
            ++m;
            last_a = (int)a;
            last_hi = k;
        }
    }
}

template <int R>
__device__ __forceinline__ uint32_t key16_at(const uint32_t (&x)[R], int p) {
    return p < R ? (x[p] & 0xFFFFu) : (x[p - R] >> 16);
}

template <int R>
__device__ __forceinline__ void scan16(const uint32_t (&x)[R], uint32_t* rec, int stride, int cap, bool write,
                                       int& m, int& last_a, int& last_hi) {
    constexpr int N = 2 * R;
    int lo = 0, prev = 0, gi = 0;
    m = 0; last_a = 0; last_hi = 0;
#pragma unroll
    for (int p = 0; p < N; ++p) {
        const uint32_t key = key16_at<R>(x, p);
        const uint32_t a = key >> 8;
        const int k = (int)(key & 0xFFu);
        const bool first = (p == 0) || ((key16_at<R>(x, p - 1) >> 8) != a);
        const bool last = (p == N - 1) || ((key16_at<R>(x, p + 1) >> 8) != a);
        gi = first ? 0 : max(gi, k - prev);
        lo = first ? k : lo;
        prev = k;
        if (key != KEY16_NONE && last) {
            if (write && m < cap) rec[m * stride] = (a << 24) | ((uint32_t)lo << 16) | ((uint32_t)k << 8) | (uint32_t)gi;
            ++m;
            last_a = (int)a;
            last_hi = k;
        }
    }
}

__device__ __forceinline__ int rr_records32(const Geo& g, const uint2* rec, int stride, int m) {
    DP5 v;
    dp_init(v);
    int pa = 0;
    for (int j = 0; j < m; ++j) {
        const uint2 r = rec[j * stride];
        const int a = (int)(r.x >> 16);
        dp_aisle(v, g, a - pa, (int)(r.x & 0xFFFFu), (int)(r.y >> 16), (int)(r.y & 0xFFFFu));
        pa = a;
    }
    return dp_final(v);
}

__device__ __forceinline__ int rr_records16(const Geo& g, const uint32_t* rec, int stride, int m) {
    DP5 v;
    dp_init(v);
    int pa = 0;
    for (int j = 0; j < m; ++j) {
        const uint32_t r = rec[j * stride];
        const int a = (int)(r >> 24);
        dp_aisle(v, g, a - pa, (int)((r >> 16) & 0xFFu), (int)((r >> 8) & 0xFFu), (int)(r & 0xFFu));
        pa = a;
    }
    return dp_final(v);
}

// Key source: with a shared slotting, keys come from the per-line table
// (16-bit or 32-bit entries); with per-plan slottings, from the plan's slot
// map via the line's SKU.
struct KeySrc {
    const int32_t* off;     // order offsets (global order book)
    const uint32_t* desc;   // per-order (first line << 8 | line count), shared memory
    const void* keys;       // per-line keys (shared slotting)
    const int32_t* skus;    // per-line SKUs (per-plan slotting)
    const int32_t* map;     // this plan's slot map (per-plan slotting)
};

// STAGED: the shared-slotting key table is the shared-memory copy (16-bit
// entries when KEY16); otherwise it is the 32-bit table in global memory.
template <bool KEY16, bool SHARED_MAP, bool STAGED>
__device__ __forceinline__ uint32_t key_of(const EvalArgs& a, const KeySrc& s, int l) {
    if constexpr (SHARED_MAP) {
        if constexpr (KEY16 && STAGED) return static_cast<const uint16_t*>(s.keys)[l];
        else if constexpr (KEY16) return key16_of(static_cast<const uint32_t*>(s.keys)[l]);
        else return static_cast<const uint32_t*>(s.keys)[l];
    } else {
        const int sku = s.skus[l];
        uint32_t k32 = KEY_BAD;
        if ((unsigned)sku >= (unsigned)a.n_sku) {
            flag(a.status, WH_STATUS_BAD_SKU);
        } else {
            const int loc = s.map[sku];
            if ((unsigned)loc >= (unsigned)a.g.n_loc) flag(a.status, WH_STATUS_BAD_LOC);
            else k32 = loc_key(a.g, loc);
        }
        if constexpr (KEY16) return key16_of(k32);
        else return k32;
    }
}

// ------------------------------------------------------------ tour bodies
// Each thread owns a column of slots in a shared-memory buffer: slot j of
// thread tid sits at [j*T + tid], one slot = two keys = one per-aisle record
// (4 bytes with 16-bit keys, 8 bytes with 32-bit keys), so columns of
// different threads never overlap.  A tour's keys are first staged in the
// column (key p in slot p/2, half p%2), loaded into registers with static
// indices for the sort, and the column is then reused for the records.  The
// gather itself is a plain loop over the tour's orders and their lines.
template <int N>
__device__ __forceinline__ void load32(const uint2* col, int T, int n, uint32_t (&x)[N]) {
#pragma unroll
    for (int p = 0; p < N; ++p) {
        const uint2 w = col[(p >> 1) * T];
        x[p] = p < n ? ((p & 1) ? w.y : w.x) : KEY_NONE;
    }
}

template <int R>
__device__ __forceinline__ void load16(const uint32_t* col, int T, int n, uint32_t (&x)[R]) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const uint32_t wl = col[(r >> 1) * T], wh = col[((r + R) >> 1) * T];
        x[r] = __byte_perm(wl, wh, (r & 1) ? 0x7632 : 0x5410) | (r < n ? 0u : 0xFFFFu) |
               (r + R < n ? 0u : 0xFFFF0000u);
    }
}

template <int N>
__device__ __forceinline__ void tour32(const EvalArgs& a, uint2* col, int T, int n, bool need_rr, int& cs,
                                       int& cr) {
    uint32_t x[N];
    load32<N>(col, T, n, x);
    bitonic_sort<N>(x);
    int m, last_a, last_hi;
    scan32<N>(x, col, T, a.max_rec, need_rr, m, last_a, last_hi);
    cs = sshape_cost(a.g, m, last_a, last_hi);
    cr = need_rr ? rr_records32(a.g, col, T, min(m, a.max_rec)) : 0;
}

template <int R>
__device__ __forceinline__ void tour16(const EvalArgs& a, uint32_t* col, int T, int n, bool need_rr, int& cs,
                                       int& cr) {
    uint32_t x[R];
    load16<R>(col, T, n, x);
    sort16x2<R>(x);
    int m, last_a, last_hi;
    scan16<R>(x, col, T, a.max_rec, need_rr, m, last_a, last_hi);
    cs = sshape_cost(a.g, m, last_a, last_hi);
    cr = need_rr ? rr_records16(a.g, col, T, min(m, a.max_rec)) : 0;
}

// Segmented sum over the lanes of a warp whose `key` (plan id, non-decreasing
// with the lane) is equal; the first lane of each segment ends up with the
// segment's total.
__device__ __forceinline__ long long segmented_sum(long long v, int key, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long ov = __shfl_down_sync(0xffffffffu, v, o);
        const int ok = __shfl_down_sync(0xffffffffu, key, o);
        if (lane + o < 32 && ok == key) v += ov;
    }
    return v;
}

// ------------------------------------------------------------------ kernels

// Per-instance staging of the order book into shared memory: one descriptor
// per order (first line << 8 | line count; count 255 marks an order that the
// short path does not take: malformed, or 255 lines or more, so its tours go
// to the long-tour kernel, which checks them) and one key (or SKU) per line.
template <bool KEY16, bool SHARED_MAP>
__device__ __forceinline__ void stage_tables(const EvalArgs& a, uint32_t* s_desc, void* s_tab, KeySrc& src,
                                             int tid, int T) {
    for (int o = tid; o < a.n_orders; o += T) {
        const int lb = a.order_off[o], le = a.order_off[o + 1];
        const bool ok = lb >= 0 && le >= lb && le <= a.n_lines && le - lb < 255 && lb < (1 << 24);
        s_desc[o] = ok ? ((uint32_t)lb << 8) | (uint32_t)(le - lb) : 0xFFu;
    }
    if constexpr (SHARED_MAP) {
        if constexpr (KEY16) {
            uint16_t* k16 = static_cast<uint16_t*>(s_tab);
            for (int i = tid; i < a.n_lines; i += T) k16[i] = (uint16_t)key16_of(a.line_key[i]);
        } else {
            uint32_t* k32 = static_cast<uint32_t*>(s_tab);
            for (int i = tid; i < a.n_lines; i += T) k32[i] = a.line_key[i];
        }
        src.keys = s_tab;
    } else {
        int32_t* sk = static_cast<int32_t*>(s_tab);
        for (int i = tid; i < a.n_lines; i += T) sk[i] = a.line_sku[i];
        src.skus = sk;
    }
    src.desc = s_desc;
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

// One warp scores the 32-tour chunks [c_begin, c_end) of instance `a`, one
// tour per lane, and adds its plans' sums with one atomic per plan segment.
template <bool KEY16, bool SHARED_MAP, bool SMEM_TABLES>
__device__ __forceinline__ void eval_chunks(const EvalArgs& a, KeySrc src, uint32_t mask, int inst, int c_begin,
                                            int c_end, uint32_t* col16, uint2* col32, int T, int lane) {
    const bool need_rr = (mask & WH_ROUTE_OPTIMAL) != 0;
    const bool want_s = (mask & WH_ROUTE_SSHAPE) != 0;
    // plan of the first tour: largest p with plan_tour_off[p] <= t
    int plan = 0;
    {
        const int t0 = c_begin * 32;
        int lo = 0, hi = a.n_plans - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.plan_tour_off[mid] <= t0) lo = mid; else hi = mid - 1;
        }
        plan = lo;
    }
    for (int c = c_begin; c < c_end; ++c) {
        const int t = c * 32 + lane;
        const bool active = t < a.n_tours;
        while (plan + 1 < a.n_plans && a.plan_tour_off[plan + 1] <= t) ++plan;
        if constexpr (!SHARED_MAP) src.map = a.slot_map + (int64_t)plan * a.slot_stride;
        // one pass over the tour's orders: check them, count the lines and
        // stage the first SHORT_MAX keys in this thread's buffer column
        int n = 0;
        bool bad = false, kbad = false;
        if (active) {
            const int q0 = __ldg(a.tour_off + t), q1 = __ldg(a.tour_off + t + 1);
            if (q0 < 0 || q1 < q0 || (int64_t)q1 > a.n_seq) {
                flag(a.status, WH_STATUS_BAD_OFFSET);
                bad = true;
            } else {
                // software-pipelined: order ids two ahead, descriptors one ahead
                int o2 = q0 + 1 < q1 ? __ldg(a.order_seq + q0 + 1) : 0;
                uint32_t d1 = 0;
                int o1 = 0;
                if (q0 < q1) {
                    o1 = __ldg(a.order_seq + q0);
                    if constexpr (SMEM_TABLES) d1 = (unsigned)o1 < (unsigned)a.n_orders ? src.desc[o1] : 0xFFFFFFFFu;
                }
                for (int q = q0; q < q1; ++q) {
                    const int o = o1;
                    const uint32_t d = d1;
                    o1 = o2;
                    if constexpr (SMEM_TABLES)
                        d1 = (q + 1 < q1 && (unsigned)o1 < (unsigned)a.n_orders) ? src.desc[o1] : 0xFFFFFFFFu;
                    o2 = q + 2 < q1 ? __ldg(a.order_seq + q + 2) : 0;
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
                    for (int l = lb; l < le; ++l, ++n) {
                        const uint32_t k = key_of<KEY16, SHARED_MAP, SMEM_TABLES>(a, src, l);
                        if constexpr (KEY16) {
                            kbad |= k == KEY16_BAD;
                            reinterpret_cast<uint16_t*>(col16 + (n >> 1) * T)[n & 1] = (uint16_t)k;
                        } else {
                            kbad |= k == KEY_BAD;
                            reinterpret_cast<uint32_t*>(col32 + (n >> 1) * T)[n & 1] = k;
                        }
                    }
                }
            }
        }
        bool is_long = active && !bad && n > SHORT_MAX;
        if (is_long && !defer_long(a, inst, t, plan)) { is_long = false; bad = true; }
        const bool run = active && !bad && !is_long;
        const int nr = run ? n : 0;
        const int nmax = __reduce_max_sync(0xffffffffu, nr);
        int cs = 0, cr = 0;
        if constexpr (KEY16) {
            if (nmax <= 16) tour16<8>(a, col16, T, nr, need_rr, cs, cr);
            else if (nmax <= 32) tour16<16>(a, col16, T, nr, need_rr, cs, cr);
            else tour16<32>(a, col16, T, nr, need_rr, cs, cr);
        } else {
            if (nmax <= 16) tour32<16>(a, col32, T, nr, need_rr, cs, cr);
            else if (nmax <= 32) tour32<32>(a, col32, T, nr, need_rr, cs, cr);
            else tour32<64>(a, col32, T, nr, need_rr, cs, cr);
        }
        const bool ok = run && !kbad;
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
    const int i0 = blockIdx.x * blockDim.x + threadIdx.x;
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

template <bool KEY16, bool SHARED_MAP, bool SMEM_TABLES>
__global__ void __launch_bounds__(256, 2) k_eval_short(EvalArgs a) {
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
    if constexpr (SMEM_TABLES) {
        stage_tables<KEY16, SHARED_MAP>(a, s_desc, s_tab, src, tid, T);
        __syncthreads();
    }
    // this warp's contiguous range of 32-tour chunks
    const int warps = gridDim.x * (T >> 5);
    const int gw = blockIdx.x * (T >> 5) + (tid >> 5);
    const int n_chunks = (a.n_tours + 31) >> 5;
    const int per = (n_chunks + warps - 1) / warps;
    const int c_begin = gw * per;
    const int c_end = min(c_begin + per, n_chunks);
    if (c_begin >= c_end) return;
    eval_chunks<KEY16, SHARED_MAP, SMEM_TABLES>(a, src, a.mask, 0, c_begin, c_end,
                                                reinterpret_cast<uint32_t*>(buf_base) + tid,
                                                reinterpret_cast<uint2*>(buf_base) + tid, T, lane);
}

// Persistent batch kernel: CTAs pop work items (instance, chunk range) from
// a queue ordered largest first, stage that instance's order book once, and
// split the item's chunks among their warps.
template <bool KEY16, bool SMEM_TABLES>
__global__ void __launch_bounds__(256, 2) k_eval_batch(BatchArgs b) {
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
            if constexpr (SMEM_TABLES) stage_tables<KEY16, true>(s_a, s_desc, s_tab, src, tid, T);
            staged = w.inst;
        }
        __syncthreads();
        const int n = w.chunk_end - w.chunk_begin;
        const int per = (n + nw - 1) / nw;
        const int cb = w.chunk_begin + warp * per;
        const int ce = min(cb + per, w.chunk_end);
        if (cb < ce) eval_chunks<KEY16, true, SMEM_TABLES>(s_a, src, b.mask, w.inst, cb, ce, col16, col32, T, lane);
        __syncthreads();
    }
}

__device__ __forceinline__ int warp_inclusive_scan(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// One warp per deferred tour (more than SHORT_MAX lines): keys gathered into
// a per-warp shared-memory buffer, bitonic-sorted there, then one lane runs
// the record scan and the DP.
template <bool SHARED_MAP>
__global__ void __launch_bounds__(LONG_WARPS * 32) k_eval_long(LongArgs L) {
    __shared__ uint32_t buf[LONG_WARPS][LONG_MAXL];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int count = min(*L.count, L.cap);
    uint32_t* kb = buf[warp];
    const bool need_rr = (L.mask & WH_ROUTE_OPTIMAL) != 0;
    const bool want_s = (L.mask & WH_ROUTE_SSHAPE) != 0;
    for (int w = blockIdx.x * LONG_WARPS + warp; w < count; w += gridDim.x * LONG_WARPS) {
        const int inst = L.list[3 * w], t = L.list[3 * w + 1], plan = L.list[3 * w + 2];
        const EvalArgs& a = L.insts ? L.insts[inst] : L.single;
        KeySrc src = global_src(a);
        const int q0 = a.tour_off[t], q1 = a.tour_off[t + 1];   // checked by the short kernel
        if constexpr (!SHARED_MAP) src.map = a.slot_map + (int64_t)plan * a.slot_stride;
        int n = 0;
        bool bad = false;
        for (int qb = q0; qb < q1; qb += 32) {
            const int q = qb + lane;
            int lb = 0, le = 0;
            if (q < q1) {
                const int o = a.order_seq[q];   // in range: checked by the short kernel
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
            int pos = n + incl - cnt;
            for (int l = lb; l < le; ++l, ++pos) {
                const uint32_t k = key_of<false, SHARED_MAP, false>(a, src, l);
                bad |= (k == KEY_BAD);
                if (pos < LONG_MAXL) kb[pos] = k;
            }
            n += __shfl_sync(0xffffffffu, incl, 31);
        }
        bad = __any_sync(0xffffffffu, bad);
        if (n > LONG_MAXL || bad) {
            if (lane == 0) {
                if (n > LONG_MAXL) flag(a.status, WH_STATUS_TOUR_TOO_LONG);
                if (a.tour_s) a.tour_s[t] = -1;
                if (a.tour_rr) a.tour_rr[t] = -1;
            }
            __syncwarp();
            continue;
        }
        int p2 = 64;
        while (p2 < n) p2 <<= 1;
        for (int i = n + lane; i < p2; i += 32) kb[i] = KEY_NONE;
        __syncwarp();
        for (int k = 2; k <= p2; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = lane; i < p2; i += 32) {
                    const int l = i ^ j;
                    if (l > i) {
                        const uint32_t x = kb[i], y = kb[l];
                        const bool up = (i & k) == 0;
                        if ((x > y) == up) { kb[i] = y; kb[l] = x; }
                    }
                }
                __syncwarp();
            }
        }
        if (lane == 0) {
            DP5 v;
            dp_init(v);
            int m = 0, pa = 0, lo = 0, prev = 0, gi = 0, last_a = 0, last_hi = 0;
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
                    ++m;
                    last_a = ai;
                    last_hi = k;
                }
            }
            const int cs = sshape_cost(a.g, m, last_a, last_hi);
            const int cr = need_rr ? dp_final(v) : 0;
            if (a.tour_s && want_s) a.tour_s[t] = cs;
            if (a.tour_rr && need_rr) a.tour_rr[t] = cr;
            if (a.plan_s && want_s)
                atomicAdd(reinterpret_cast<unsigned long long*>(&a.plan_s[plan]), (unsigned long long)cs);
            if (a.plan_rr && need_rr)
                atomicAdd(reinterpret_cast<unsigned long long*>(&a.plan_rr[plan]), (unsigned long long)cr);
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

template <bool K16, bool SM>
cudaError_t launch_batch_t(const BatchArgs& b, const Tuning& t, size_t smem, int num_sms, cudaStream_t s) {
    auto kern = k_eval_batch<K16, SM>;
    int grid = 0;
    cudaError_t e = grid_for(kern, t.threads, smem, num_sms, b.n_items, &grid);
    if (e != cudaSuccess) return e;
    kern<<<grid, t.threads, smem, s>>>(b);
    return cudaGetLastError();
}

}  // namespace

bool key16_ok(const Geo& g) { return g.A <= 255 && g.L <= 256; }


static size_t buffer_bytes(bool k16, int max_rec, int threads) {
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

cudaError_t launch_prep(const EvalArgs& a, cudaStream_t s) {
    int work = a.n_plans;
    if (a.line_key && a.n_lines > work) work = a.n_lines;
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

cudaError_t launch_eval_short(const EvalArgs& a, const Tuning& t, int num_sms, cudaStream_t s, int* grid_out) {
    if (t.threads % 32 != 0 || t.threads > 256 || t.threads < 32) return cudaErrorInvalidValue;
    if (a.n_tours == 0) return cudaSuccess;
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
    if (t.threads % 32 != 0 || t.threads > 256 || t.threads < 32) return cudaErrorInvalidValue;
    if (b.n_items == 0) return cudaSuccess;
    const size_t smem = eval_batch_smem_bytes(b, t, k16);
    const bool sm = t.smem_tables != 0;
    if (k16) return sm ? launch_batch_t<true, true>(b, t, smem, num_sms, s) : launch_batch_t<true, false>(b, t, smem, num_sms, s);
    return sm ? launch_batch_t<false, true>(b, t, smem, num_sms, s) : launch_batch_t<false, false>(b, t, smem, num_sms, s);
}

cudaError_t launch_eval_long(const LongArgs& L, bool shared_map, int num_sms, cudaStream_t s) {
    const int grid = num_sms * 2;
    if (shared_map) k_eval_long<true><<<grid, LONG_WARPS * 32, 0, s>>>(L);
    else k_eval_long<false><<<grid, LONG_WARPS * 32, 0, s>>>(L);
    return cudaGetLastError();
}

}  // namespace wh
