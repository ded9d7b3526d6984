// Device building blocks of a tour's cost, shared by the plan-evaluation and
// move-evaluation kernels: pick keys, the sorting networks, the per-aisle
// record scan, the S-shape closed form and the Ratliff-Rosenthal DP (Sec. 5,
// Eq. (2)).  Included by each kernel translation unit; everything lives in an
// unnamed namespace, so each unit gets its own copy.
#pragma once
#include <cuda_bf16.h>

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

// location (0 <= loc < n_loc) -> aisle << 16 | slot index; the division by 2L
// is the multiply-high form set up in Geo (one multiply and one shift)
__device__ __forceinline__ uint32_t loc_key(const Geo& g, int loc) {
    const int two_l = 2 * g.L;
    const int a = (int)(__umulhi((uint32_t)loc, g.div_m) >> g.div_s);
    const int r = loc - a * two_l;          // side*L + k
    const int k = r >= g.L ? r - g.L : r;
    return ((uint32_t)a << 16) | (uint32_t)k;
}

// 32-bit key -> 16-bit key (aisle<<8 | slot); valid when A <= 255, L <= 256
__device__ __forceinline__ uint32_t key16_of(uint32_t k32) {
    if (k32 == KEY_BAD) return KEY16_BAD;
    return ((k32 >> 8) & 0xFF00u) | (k32 & 0xFFu);
}

// 32-bit shared-window addresses for the per-line loops: one 32-bit add per
// address step instead of generic 64-bit pointer arithmetic.  Loads and
// stores are volatile with a memory clobber, so the compiler keeps them in
// order with each other and with the surrounding code's memory accesses (a
// thread's column is written, read back and rewritten in every chunk).
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

template <typename K>
__device__ __forceinline__ uint32_t lds_key(uint32_t addr) {
    if constexpr (sizeof(K) == 2) {
        unsigned short v;
        asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(addr) : "memory");
        return v;
    } else {
        uint32_t v;
        asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
        return v;
    }
}

template <typename K>
__device__ __forceinline__ void sts_key(uint32_t addr, uint32_t v) {
    if constexpr (sizeof(K) == 2)
        asm volatile("st.shared.u16 [%0], %1;" ::"r"(addr), "h"((unsigned short)v) : "memory");
    else
        asm volatile("st.shared.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// Predicated forms (no branch around the access): the load leaves its
// result undefined and the store writes nothing when p is false.
template <typename K>
__device__ __forceinline__ uint32_t lds_key_if(bool p, uint32_t addr) {
    if constexpr (sizeof(K) == 2) {
        unsigned short v;
        asm volatile("{ .reg .pred q; setp.ne.b32 q, %2, 0; @q ld.shared.u16 %0, [%1]; }"
                     : "=h"(v) : "r"(addr), "r"((uint32_t)p) : "memory");
        return v;
    } else {
        uint32_t v;
        asm volatile("{ .reg .pred q; setp.ne.b32 q, %2, 0; @q ld.shared.u32 %0, [%1]; }"
                     : "=r"(v) : "r"(addr), "r"((uint32_t)p) : "memory");
        return v;
    }
}

template <typename K>
__device__ __forceinline__ void sts_key_if(bool p, uint32_t addr, uint32_t v) {
    if constexpr (sizeof(K) == 2)
        asm volatile("{ .reg .pred q; setp.ne.b32 q, %2, 0; @q st.shared.u16 [%0], %1; }"
                     ::"r"(addr), "h"((unsigned short)v), "r"((uint32_t)p) : "memory");
    else
        asm volatile("{ .reg .pred q; setp.ne.b32 q, %2, 0; @q st.shared.u32 [%0], %1; }"
                     ::"r"(addr), "r"(v), "r"((uint32_t)p) : "memory");
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

// The same step in relative form, for the record DPs of the evaluation
// kernels: every state holds its value minus 2P * (aisle of the last step),
// so crossing d aisle gaps adds nothing to the classes whose edge pattern
// uses each gap twice (UU, E0, OE; EE switching to E0 / OE) and 2P * d to
// those that use it four times (EE, E2); the caller adds 2P * (last aisle)
// back at the end.  The vertical options are precomputed multiply-adds:
// cB = 2(Y - y_lo), cF = 2 y_hi, and leaving out the largest gap
// max(y_lo, gi*S, Y - y_hi) costs 2Y - 2*max(...) = min(cB, 2Y - 2 gi*S, cF).
// Integer arithmetic throughout, so the result equals dp_aisle's exactly.
struct DPConst {
    int p2, s2, cb0, cf0, y, y2;   // 2P, 2S, 2(Y - h), 2h, Y, 2Y
};

__device__ __forceinline__ DPConst dp_const(const Geo& g) {
    DPConst c;
    c.p2 = 2 * g.P;
    c.s2 = 2 * g.S;
    c.cb0 = 2 * (g.Y - g.h);
    c.cf0 = 2 * g.h;
    c.y = g.Y;
    c.y2 = 2 * g.Y;
    return c;
}

__device__ __forceinline__ void dp_aisle_rel(DP5& v, const DPConst& c, int d, int lo, int hi, int gi) {
    const int h2 = c.p2 * d;
    const int he0 = min(v.e0, v.ee), hoe = min(v.oe, v.ee);
    const int hee = v.ee + h2, he2 = v.e2 + h2;
    const int cB = c.cb0 - lo * c.s2, cF = c.cf0 + hi * c.s2;
    const int cG = __vimin3_s32(cB, c.y2 - gi * c.s2, cF);
    const int m3 = __vimin3_s32(he0, hoe, he2);
    const int huu = v.uu;
    v.uu = __viaddmin_s32(huu, cG, min(m3, hee) + c.y);
    v.ee = __viaddmin_s32(huu, c.y, __viaddmin_s32(m3, c.y2, hee + cG));
    v.e0 = he0 + cF;
    v.oe = hoe + cB;
    v.e2 = m3 + cG;
}

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
// Sorted keys -> per-aisle records (at most cap of them, written from the
// shared-memory address rec_sa on, stride_b bytes apart) and the S-shape
// inputs (pick-aisle count, rightmost aisle, its deepest slot).  On sorted
// keys the aisle changes between positions p and p + 1 exactly when
// key(p + 1) > (key(p) | slot mask); the padding (all ones) and the bad-key
// marker (all ones but the lowest bit) never satisfy that against their
// successor, so only the final position needs the padding test.
template <int N>
__device__ __forceinline__ void scan32(const uint32_t (&x)[N], uint32_t rec_sa, uint32_t stride_b, int cap,
                                       bool write, int& m, int& last_a, int& last_hi) {
    const uint32_t rec_end = rec_sa + stride_b * (uint32_t)cap;
    uint32_t lo = 0, gi = 0, last_key = 0;
    m = 0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const uint32_t key = x[i];
        const bool first = (i == 0) || key > (x[i - 1] | 0xFFFFu);
        const bool last = (i == N - 1) ? key != KEY_NONE : x[i + 1] > (key | 0xFFFFu);
        if (i > 0) gi = first ? 0u : max(gi, key - x[i - 1]);
        lo = first ? key : lo;
        if (last) {
            if (write && rec_sa < rec_end)
                asm volatile("st.shared.v2.u32 [%0], {%1, %2};" ::"r"(rec_sa), "r"(lo), "r"((key << 16) | gi)
                             : "memory");
            rec_sa += stride_b;
            ++m;
            last_key = key;
        }
    }
    last_a = (int)(last_key >> 16);
    last_hi = (int)(last_key & 0xFFFFu);
}

template <int R>
__device__ __forceinline__ uint32_t key16_at(const uint32_t (&x)[R], int p) {
    return p < R ? (x[p] & 0xFFFFu) : (x[p - R] >> 16);
}

template <int R>
__device__ __forceinline__ void scan16(const uint32_t (&x)[R], uint32_t rec_sa, uint32_t stride_b, int cap,
                                       bool write, int& m, int& last_a, int& last_hi) {
    constexpr int N = 2 * R;
    const uint32_t rec_end = rec_sa + stride_b * (uint32_t)cap;
    uint32_t lo = 0, gi = 0, last_key = 0;
    m = 0;
#pragma unroll
    for (int p = 0; p < N; ++p) {
        const uint32_t key = key16_at<R>(x, p);
        const bool first = (p == 0) || key > (key16_at<R>(x, p - 1) | 0xFFu);
        const bool last = (p == N - 1) ? key != KEY16_NONE : key16_at<R>(x, p + 1) > (key | 0xFFu);
        if (p > 0) gi = first ? 0u : max(gi, key - key16_at<R>(x, p - 1));
        lo = first ? key : lo;
        if (last) {
            // record: aisle << 24 | shallowest slot << 16 | deepest slot << 8 | largest gap
            if (write && rec_sa < rec_end)
                sts_key<uint32_t>(rec_sa, (lo << 16) | ((key & 0xFFu) << 8) | gi);
            rec_sa += stride_b;
            ++m;
            last_key = key;
        }
    }
    last_a = (int)(last_key >> 8);
    last_hi = (int)(last_key & 0xFFu);
}

// records anywhere in memory (the long-tour passes' global scratch)
__device__ __forceinline__ int rr_records32_mem(const Geo& g, const uint2* rec, int64_t stride, int m) {
    const DPConst c = dp_const(g);
    DP5 v;
    dp_init(v);
    int pa = 0;
    // four records' loads in flight ahead of their DP steps
    for (int j0 = 0; j0 < m; j0 += 4) {
        uint2 r[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) r[u] = j0 + u < m ? rec[(j0 + u) * stride] : make_uint2(0u, 0u);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (j0 + u >= m) break;
            const int a = (int)(r[u].x >> 16);
            dp_aisle_rel(v, c, a - pa, (int)(r[u].x & 0xFFFFu), (int)(r[u].y >> 16), (int)(r[u].y & 0xFFFFu));
            pa = a;
        }
    }
    return dp_final(v) + c.p2 * pa;
}

__device__ __forceinline__ int rr_records32(const Geo& g, uint32_t rec_sa, uint32_t stride_b, int m) {
    const DPConst c = dp_const(g);
    DP5 v;
    dp_init(v);
    int pa = 0;
    for (int j = 0; j < m; ++j, rec_sa += stride_b) {
        uint32_t rx, ry;
        asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(rx), "=r"(ry) : "r"(rec_sa) : "memory");
        const int a = (int)(rx >> 16);
        dp_aisle_rel(v, c, a - pa, (int)(rx & 0xFFFFu), (int)(ry >> 16), (int)(ry & 0xFFFFu));
        pa = a;
    }
    return dp_final(v) + c.p2 * pa;
}

__device__ __forceinline__ int rr_records16(const Geo& g, uint32_t rec_sa, uint32_t stride_b, int m) {
    const DPConst c = dp_const(g);
    DP5 v;
    dp_init(v);
    int pa = 0;
    for (int j = 0; j < m; ++j, rec_sa += stride_b) {
        const uint32_t r = lds_key<uint32_t>(rec_sa);
        const int a = (int)(r >> 24);
        dp_aisle_rel(v, c, a - pa, (int)((r >> 16) & 0xFFu), (int)((r >> 8) & 0xFFu), (int)(r & 0xFFu));
        pa = a;
    }
    return dp_final(v) + c.p2 * pa;
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
__device__ __forceinline__ void load32(uint32_t col_sa, uint32_t slot_b, int n, uint32_t (&x)[N]) {
#pragma unroll
    for (int p = 0; p < N; p += 2) {
        uint32_t wx, wy;
        asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];"
                     : "=r"(wx), "=r"(wy)
                     : "r"(col_sa + (uint32_t)(p >> 1) * slot_b)
                     : "memory");
        x[p] = p < n ? wx : KEY_NONE;
        if (p + 1 < N) x[p + 1] = p + 1 < n ? wy : KEY_NONE;
    }
}

template <int R>
__device__ __forceinline__ void load16(uint32_t col_sa, uint32_t slot_b, int n, uint32_t (&x)[R]) {
    uint32_t wv[R];
#pragma unroll
    for (int j = 0; j < R; ++j) wv[j] = lds_key<uint32_t>(col_sa + (uint32_t)j * slot_b);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const uint32_t wl = wv[r >> 1], wh = wv[(r + R) >> 1];
        x[r] = __byte_perm(wl, wh, (r & 1) ? 0x7632 : 0x5410) | (r < n ? 0u : 0xFFFFu) |
               (r + R < n ? 0u : 0xFFFF0000u);
    }
}

// m: the tour's pick-aisle count; with the optimal rule, a tour of more
// than a.max_rec pick aisles has no room for its records: cr is then not its
// cost and the caller hands the tour to a long-tour pass.  With check set,
// *kbad reports whether one of the n keys is the bad-key marker (a line whose
// SKU or slot is invalid), tested on the loaded registers two keys at a time.
template <int N>
__device__ __forceinline__ void tour32(const EvalArgs& a, uint2* col, int T, int n, bool need_rr, int& cs,
                                       int& cr, int& m, bool check = false, bool* kbad = nullptr) {
    const uint32_t col_sa = smem_addr(col), slot_b = 8u * (uint32_t)T;
    uint32_t x[N];
    load32<N>(col_sa, slot_b, n, x);
    if (check) {
        bool b = false;
#pragma unroll
        for (int p = 0; p < N; ++p) b |= x[p] == KEY_BAD;
        *kbad = b;
    }
    bitonic_sort<N>(x);
    int last_a, last_hi;
    scan32<N>(x, col_sa, slot_b, a.max_rec, need_rr, m, last_a, last_hi);
    cs = sshape_cost(a.g, m, last_a, last_hi);
    cr = need_rr ? rr_records32(a.g, col_sa, slot_b, min(m, a.max_rec)) : 0;
}

template <int R>
__device__ __forceinline__ void tour16(const EvalArgs& a, uint32_t* col, int T, int n, bool need_rr, int& cs,
                                       int& cr, int& m, bool check = false, bool* kbad = nullptr) {
    const uint32_t col_sa = smem_addr(col), slot_b = 4u * (uint32_t)T;
    uint32_t x[R];
    load16<R>(col_sa, slot_b, n, x);
    if (check) {
        uint32_t acc = 0u;
#pragma unroll
        for (int r = 0; r < R; ++r) acc |= __vcmpeq2(x[r], (KEY16_BAD << 16) | KEY16_BAD);
        *kbad = acc != 0u;
    }
    sort16x2<R>(x);
    int last_a, last_hi;
    scan16<R>(x, col_sa, slot_b, a.max_rec, need_rr, m, last_a, last_hi);
    cs = sshape_cost(a.g, m, last_a, last_hi);
    cr = need_rr ? rr_records16(a.g, col_sa, slot_b, min(m, a.max_rec)) : 0;
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

// Bitonic sort of the 32 * KPL keys kb[0..32*KPL) held KPL per lane (lane
// holds elements KPL*lane .. KPL*lane + KPL-1): partners at distance < KPL
// are in the lane's own registers, farther ones in lane ^ (d / KPL) (one
// shuffle).  Sorted keys are written back to kb.
template <int KPL>
__device__ __forceinline__ void warp_sort_keys(uint32_t* kb, int lane) {
    uint32_t x[KPL];
#pragma unroll
    for (int j = 0; j < KPL; ++j) x[j] = kb[KPL * lane + j];
#pragma unroll
    for (int k = 2; k <= 32 * KPL; k <<= 1) {
#pragma unroll
        for (int d = k >> 1; d > 0; d >>= 1) {
            if (d < KPL) {
#pragma unroll
                for (int j = 0; j < KPL; ++j) {
                    const int jp = j ^ d;
                    if (jp > j) {
                        const int e = KPL * lane + j;
                        const bool asc = (e & k) == 0;
                        const uint32_t lo = min(x[j], x[jp]), hi = max(x[j], x[jp]);
                        x[j] = asc ? lo : hi;
                        x[jp] = asc ? hi : lo;
                    }
                }
            } else {
#pragma unroll
                for (int j = 0; j < KPL; ++j) {
                    const int e = KPL * lane + j;
                    const uint32_t other = __shfl_xor_sync(0xffffffffu, x[j], d / KPL);
                    const bool lower = (e & d) == 0, asc = (e & k) == 0;
                    x[j] = (lower == asc) ? min(x[j], other) : max(x[j], other);
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < KPL; ++j) kb[KPL * lane + j] = x[j];
}

// Sort kb[0..n) ascending (n <= LONG_MAXL) by one warp: padded with KEY_NONE
// to a power of two >= 64; up to 256 keys in registers (warp_sort_keys),
// longer runs by a bitonic network in shared memory.
__device__ __forceinline__ void warp_sort_buffer(uint32_t* kb, int n, int lane) {
    int p2 = 64;
    while (p2 < n) p2 <<= 1;
    for (int x = n + lane; x < p2; x += 32) kb[x] = KEY_NONE;
    __syncwarp();
    if (p2 == 64) {
        warp_sort_keys<2>(kb, lane);
    } else if (p2 == 128) {
        warp_sort_keys<4>(kb, lane);
    } else if (p2 == 256) {
        warp_sort_keys<8>(kb, lane);
    } else {
        for (int k = 2; k <= p2; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int x = lane; x < p2; x += 32) {
                    const int l = x ^ j;
                    if (l > x) {
                        const uint32_t u = kb[x], v = kb[l];
                        const bool up = (x & k) == 0;
                        if ((u > v) == up) {
                            kb[x] = v;
                            kb[l] = u;
                        }
                    }
                }
                __syncwarp();
            }
        }
    }
    __syncwarp();
}

// inclusive prefix sum over the 32 lanes of a warp
__device__ __forceinline__ int warp_inclusive_scan(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

}  // namespace
}  // namespace wh
