// Plan evaluation kernels for sm_103a.
//
// What is computed (Sec. 5, Eq. (2)): for every tour, the length of the
// S-shape route and of the optimal route through its picks, and for every
// plan the int64 sum of its tours' lengths.
//
// Design (one GPU, integer work, no tensor-core shape):
//   k_line_keys   -- layout/slot-map build: one packed key (aisle<<16 | slot)
//                    per order line under the shared slotting.
//   k_eval_short  -- one tour per thread for tours of <= 64 lines: keys are
//                    gathered into registers, sorted by a bitonic network
//                    fully unrolled over registers, reduced to per-aisle
//                    records (aisle, shallowest and deepest pick, largest
//                    gap between consecutive picks) kept in shared memory,
//                    then the S-shape closed form and the optimal-route DP
//                    run over the records.  Per-plan int64 sums are
//                    accumulated in shared memory and stored once per plan.
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
constexpr int LONG_WARPS = 4;
constexpr int LONG_MAXL = WH_MAX_TOUR_LINES;
constexpr int SHORT_THREADS_MAX = 256;

__device__ __forceinline__ void flag(uint32_t* status, uint32_t bit) { atomicOr(status, bit); }

__device__ __forceinline__ uint32_t loc_key(const Geo& g, int loc) {
    const int two_l = 2 * g.L;
    const int a = loc / two_l;
    const int r = loc - a * two_l;          // side*L + k
    const int k = r >= g.L ? r - g.L : r;
    return ((uint32_t)a << 16) | (uint32_t)k;
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
__device__ __forceinline__ void dp_aisle(DP5& v, const Geo& g, int d, int lo, int hi, int gi) {
    // cross the d aisle gaps: (1,1) for UU; (2,0) / (0,2) for E0 / OE, which
    // EE may also switch to; (2,2) for EE and E2
    const int h2 = 2 * g.P * d, h4 = 2 * h2;
    const int huu = v.uu + h2;
    const int he0 = min(v.e0, v.ee) + h2;
    const int hoe = min(v.oe, v.ee) + h2;
    const int hee = v.ee + h4;
    const int he2 = v.e2 + h4;
    // vertical options of this aisle: traverse Y, double traverse 2Y, leave
    // out the largest gap 2(Y-g), from the back 2(Y-y_lo), from the front 2*y_hi
    const int ylo = g.h + lo * g.S, yhi = g.h + hi * g.S;
    const int gap = max(max(ylo, gi * g.S), g.Y - yhi);
    const int cG = 2 * (g.Y - gap), cB = 2 * (g.Y - ylo), cF = 2 * yhi;
    const int cT = g.Y, cD = 2 * g.Y;
    const int m3 = min(min(he0, hoe), he2);
    v.uu = min(min(huu + cG, min(m3, hee) + cT), INF);
    v.ee = min(min(min(huu + cT, m3 + cD), hee + cG), INF);
    v.e0 = min(he0 + cF, INF);
    v.oe = min(hoe + cB, INF);
    v.e2 = min(m3 + cG, INF);
}

__device__ __forceinline__ int dp_final(const DP5& v) { return min(min(v.ee, v.e0), v.oe); }

// S-shape closed form from the number of pick aisles m, the rightmost pick
// aisle and its deepest slot.
__device__ __forceinline__ int sshape_cost(const Geo& g, int m, int last_a, int last_hi) {
    if (m == 0) return 0;
    const int d_r = g.h + last_hi * g.S;
    return 2 * last_a * g.P + ((m & 1) ? (m - 1) * g.Y + 2 * d_r : m * g.Y);
}

// ---------------------------------------------------------- register sort
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

// Sorted keys -> per-aisle records (written to rec[j*stride], at most cap of
// them), plus the S-shape inputs.
template <int N>
__device__ __forceinline__ void scan_records(const uint32_t (&x)[N], uint2* rec, int stride, int cap,
                                             bool write, int& m, int& last_a, int& last_hi) {
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

__device__ __forceinline__ int rr_records(const Geo& g, const uint2* rec, int stride, int m) {
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

// key of line l for the tour's slotting
template <bool SHARED_MAP>
__device__ __forceinline__ uint32_t key_of(const EvalArgs& a, const uint32_t* keys, const int32_t* skus,
                                           const int32_t* map, int l) {
    if constexpr (SHARED_MAP) {
        return keys[l];
    } else {
        const int sku = skus[l];
        if ((unsigned)sku >= (unsigned)a.n_sku) { flag(a.status, WH_STATUS_BAD_SKU); return KEY_BAD; }
        const int loc = map[sku];
        if ((unsigned)loc >= (unsigned)a.g.n_loc) { flag(a.status, WH_STATUS_BAD_LOC); return KEY_BAD; }
        return loc_key(a.g, loc);
    }
}

template <int N, bool SHARED_MAP>
__device__ __forceinline__ void short_tour(const EvalArgs& a, const int32_t* off, const uint32_t* keys,
                                           const int32_t* skus, const int32_t* map, int q0, int q1,
                                           uint2* rec, bool need_rr, int& cs, int& cr, bool& bad) {
    uint32_t x[N];
    int q = q0, l = 0, le = 0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        while (l >= le && q < q1) {
            const int o = a.order_seq[q++];
            l = off[o];
            le = off[o + 1];
        }
        uint32_t k = KEY_NONE;
        if (l < le) { k = key_of<SHARED_MAP>(a, keys, skus, map, l); ++l; }
        bad |= (k == KEY_BAD);
        x[i] = k;
    }
    bitonic_sort<N>(x);
    int m, last_a, last_hi;
    scan_records<N>(x, rec, blockDim.x, a.max_rec, need_rr, m, last_a, last_hi);
    cs = sshape_cost(a.g, m, last_a, last_hi);
    cr = need_rr ? rr_records(a.g, rec, blockDim.x, min(m, a.max_rec)) : 0;
}

// ------------------------------------------------------------------ kernels

__global__ void k_line_keys(EvalArgs a, uint32_t* line_key) {
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < a.n_lines; l += gridDim.x * blockDim.x) {
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

template <bool SMEM_TABLES, bool SHARED_MAP>
__global__ void __launch_bounds__(128, 4) k_eval_short(EvalArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int T = blockDim.x, tid = threadIdx.x;
    const int K = a.plans_per_item;
    unsigned long long* acc = reinterpret_cast<unsigned long long*>(smem);   // [2K]
    uint2* rec_all = reinterpret_cast<uint2*>(acc + 2 * K);                   // [max_rec][T]
    int32_t* s_off = reinterpret_cast<int32_t*>(rec_all + (size_t)a.max_rec * T);
    int32_t* s_tab = s_off + a.n_orders + 1;  // line keys (shared map) or SKUs
    uint2* rec = rec_all + tid;

    const int32_t* off = a.order_off;
    const uint32_t* keys = a.line_key;
    const int32_t* skus = a.line_sku;
    if constexpr (SMEM_TABLES) {
        for (int i = tid; i <= a.n_orders; i += T) s_off[i] = a.order_off[i];
        if constexpr (SHARED_MAP) {
            for (int i = tid; i < a.n_lines; i += T) s_tab[i] = (int32_t)a.line_key[i];
            keys = reinterpret_cast<const uint32_t*>(s_tab);
        } else {
            for (int i = tid; i < a.n_lines; i += T) s_tab[i] = a.line_sku[i];
            skus = s_tab;
        }
        off = s_off;
        __syncthreads();
    }
    const bool need_rr = (a.mask & WH_ROUTE_OPTIMAL) != 0;

    for (int item = blockIdx.x; item < a.n_items; item += gridDim.x) {
        const int p0 = item * K;
        const int p1 = min(p0 + K, a.n_plans);
        int T0 = a.plan_tour_off[p0];
        int T1 = a.plan_tour_off[p1];
        if (T0 < 0 || T1 < T0 || T1 > a.n_tours) {
            if (tid == 0) flag(a.status, WH_STATUS_BAD_OFFSET);
            T1 = T0 = 0;
        }
        for (int i = tid; i < 2 * K; i += T) acc[i] = 0ull;
        __syncthreads();
        for (int c = T0; c < T1; c += T) {
            const int t = c + tid;
            const bool active = t < T1;
            int plan = p0;
            int q0 = 0, q1 = 0, n = 0;
            bool bad = false;
            if (active) {
                while (plan + 1 < p1 && a.plan_tour_off[plan + 1] <= t) ++plan;
                q0 = a.tour_off[t];
                q1 = a.tour_off[t + 1];
                if (q0 < 0 || q1 < q0 || (int64_t)q1 > a.n_seq) {
                    flag(a.status, WH_STATUS_BAD_OFFSET);
                    bad = true;
                } else {
                    for (int q = q0; q < q1; ++q) {
                        const int o = a.order_seq[q];
                        if ((unsigned)o >= (unsigned)a.n_orders) { flag(a.status, WH_STATUS_BAD_ORDER); bad = true; break; }
                        const int lb = off[o], le = off[o + 1];
                        if (lb < 0 || le < lb || le > a.n_lines) { flag(a.status, WH_STATUS_BAD_OFFSET); bad = true; break; }
                        n += le - lb;
                    }
                }
            }
            const bool is_long = active && !bad && n > SHORT_MAX;
            if (is_long) {
                const int slot = atomicAdd(a.long_count, 1);
                a.long_list[2 * slot] = t;
                a.long_list[2 * slot + 1] = plan;
            }
            const bool run = active && !bad && !is_long;
            if (!run) q1 = q0;   // gather nothing
            const int nmax = __reduce_max_sync(0xffffffffu, run ? n : 0);
            const int32_t* map = SHARED_MAP ? nullptr : a.slot_map + (int64_t)plan * a.slot_stride;
            int cs = 0, cr = 0;
            bool kbad = false;
            if (nmax <= 16) short_tour<16, SHARED_MAP>(a, off, keys, skus, map, q0, q1, rec, need_rr, cs, cr, kbad);
            else if (nmax <= 32) short_tour<32, SHARED_MAP>(a, off, keys, skus, map, q0, q1, rec, need_rr, cs, cr, kbad);
            else short_tour<64, SHARED_MAP>(a, off, keys, skus, map, q0, q1, rec, need_rr, cs, cr, kbad);
            if (active && (bad || kbad)) {
                if (a.tour_s) a.tour_s[t] = -1;
                if (a.tour_rr) a.tour_rr[t] = -1;
            } else if (run) {
                if (a.tour_s && (a.mask & WH_ROUTE_SSHAPE)) a.tour_s[t] = cs;
                if (a.tour_rr && need_rr) a.tour_rr[t] = cr;
                atomicAdd(&acc[2 * (plan - p0)], (unsigned long long)cs);
                atomicAdd(&acc[2 * (plan - p0) + 1], (unsigned long long)cr);
            }
        }
        __syncthreads();
        for (int q = tid; q < p1 - p0; q += T) {
            if (a.plan_s && (a.mask & WH_ROUTE_SSHAPE)) a.plan_s[p0 + q] = (int64_t)acc[2 * q];
            if (a.plan_rr && need_rr) a.plan_rr[p0 + q] = (int64_t)acc[2 * q + 1];
        }
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

template <bool SHARED_MAP>
__global__ void __launch_bounds__(LONG_WARPS * 32) k_eval_long(EvalArgs a) {
    __shared__ uint32_t buf[LONG_WARPS][LONG_MAXL];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int count = *a.long_count;
    uint32_t* kb = buf[warp];
    const bool need_rr = (a.mask & WH_ROUTE_OPTIMAL) != 0;
    for (int w = blockIdx.x * LONG_WARPS + warp; w < count; w += gridDim.x * LONG_WARPS) {
        const int t = a.long_list[2 * w], plan = a.long_list[2 * w + 1];
        const int q0 = a.tour_off[t], q1 = a.tour_off[t + 1];   // checked by k_eval_short
        const int32_t* map = SHARED_MAP ? nullptr : a.slot_map + (int64_t)plan * a.slot_stride;
        int n = 0;
        bool bad = false;
        for (int qb = q0; qb < q1; qb += 32) {
            const int q = qb + lane;
            int lb = 0, le = 0;
            if (q < q1) {
                const int o = a.order_seq[q];
                lb = a.order_off[o];
                le = a.order_off[o + 1];
            }
            const int cnt = le - lb;
            const int incl = warp_inclusive_scan(cnt);
            int pos = n + incl - cnt;
            for (int l = lb; l < le; ++l, ++pos) {
                const uint32_t k = key_of<SHARED_MAP>(a, a.line_key, a.line_sku, map, l);
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
            if (a.tour_s && (a.mask & WH_ROUTE_SSHAPE)) a.tour_s[t] = cs;
            if (a.tour_rr && need_rr) a.tour_rr[t] = cr;
            if (a.plan_s && (a.mask & WH_ROUTE_SSHAPE))
                atomicAdd(reinterpret_cast<unsigned long long*>(&a.plan_s[plan]), (unsigned long long)cs);
            if (a.plan_rr && need_rr)
                atomicAdd(reinterpret_cast<unsigned long long*>(&a.plan_rr[plan]), (unsigned long long)cr);
        }
        __syncwarp();
    }
}

template <bool SM, bool SH>
cudaError_t set_smem(size_t bytes) {
    return cudaFuncSetAttribute(k_eval_short<SM, SH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <bool SM, bool SH>
cudaError_t launch_short_t(const EvalArgs& a, const Tuning& t, size_t smem, int num_sms, cudaStream_t s,
                           int* grid_out) {
    cudaError_t e = set_smem<SM, SH>(smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_eval_short<SM, SH>, t.threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int grid = per_sm * num_sms;
    if (grid > a.n_items) grid = a.n_items;
    if (grid < 1) grid = 1;
    if (grid_out) *grid_out = grid;
    k_eval_short<SM, SH><<<grid, t.threads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

size_t eval_short_smem_bytes(const EvalArgs& a, const Tuning& t) {
    size_t b = sizeof(unsigned long long) * 2 * (size_t)t.plans_per_item;
    b += sizeof(uint2) * (size_t)a.max_rec * (size_t)t.threads;
    if (t.smem_tables) b += sizeof(int32_t) * ((size_t)a.n_orders + 1 + (size_t)a.n_lines);
    return b;
}

cudaError_t launch_line_keys(const EvalArgs& a, uint32_t* line_key, cudaStream_t s) {
    if (a.n_lines <= 0) return cudaSuccess;
    int grid = (a.n_lines + 255) / 256;
    if (grid > 4096) grid = 4096;
    k_line_keys<<<grid, 256, 0, s>>>(a, line_key);
    return cudaGetLastError();
}

cudaError_t launch_eval_short(const EvalArgs& a, const Tuning& t, int num_sms, cudaStream_t s, int* grid_out) {
    if (t.threads % 32 != 0 || t.threads > SHORT_THREADS_MAX || t.threads < 32) return cudaErrorInvalidValue;
    const size_t smem = eval_short_smem_bytes(a, t);
    const bool shared_map = a.slot_stride == 0;
    if (t.smem_tables) {
        return shared_map ? launch_short_t<true, true>(a, t, smem, num_sms, s, grid_out)
                          : launch_short_t<true, false>(a, t, smem, num_sms, s, grid_out);
    }
    return shared_map ? launch_short_t<false, true>(a, t, smem, num_sms, s, grid_out)
                      : launch_short_t<false, false>(a, t, smem, num_sms, s, grid_out);
}

cudaError_t launch_eval_long(const EvalArgs& a, int num_sms, cudaStream_t s) {
    const int grid = num_sms * 2;
    if (a.slot_stride == 0) k_eval_long<true><<<grid, LONG_WARPS * 32, 0, s>>>(a);
    else k_eval_long<false><<<grid, LONG_WARPS * 32, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace wh
