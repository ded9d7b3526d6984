// Move-delta kernels for sm_103a: the change of a plan's S-shape and optimal
// costs under a neighbourhood move (Sec. 5: subroutine 4 evaluates a change of
// product position; the picking list decides which orders share a tour).
//
// Only the tours a move changes are re-costed:
//   order swap (o1, o2)     -> the two tours holding them, each with one order
//                              exchanged;
//   relocate (o, tour)      -> the source tour without o, the target with o;
//   SKU-slot swap (s1, s2)  -> every tour holding an order with s1 or s2,
//                              under the plan's slotting with the two
//                              locations exchanged.
// Pipeline: per-tour line counts and the plan's order -> tour map; the SKU ->
// orders index of the order book; per move a check, a status and a task count;
// an exclusive scan of the counts; the task list; one task per thread (tasks
// over SHORT_MAX lines: one warp each) re-costing one changed tour and adding
// (new - old) into the move's two int64 deltas.  A SKU-swap move lists one task
// per (order with s1 or s2); of the tasks that land in the same tour only the
// one of the smallest such order counts, so no de-duplication pass is needed.
#include "tour_core.cuh"
#include "feat_core.cuh"

namespace wh {

namespace {

constexpr int MV_THREADS = 128;

__device__ __forceinline__ int order_lines_checked(const EvalArgs& a, int o, int& lb, int& le) {
    if ((unsigned)o >= (unsigned)a.n_orders) return -1;
    lb = a.order_off[o];
    le = a.order_off[o + 1];
    if (lb < 0 || le < lb || le > a.n_lines) return -1;
    return le - lb;
}

// plan of global tour t: largest p with plan_tour_off[p] <= t
__device__ __forceinline__ int plan_of_tour(const EvalArgs& a, int t) {
    int lo = 0, hi = a.n_plans - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.plan_tour_off[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void k_mv_tours(MoveArgs M) {
    const EvalArgs& a = M.a;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < a.n_tours; t += gridDim.x * blockDim.x) {
        const int p = plan_of_tour(a, t);
        const int q0 = a.tour_off[t], q1 = a.tour_off[t + 1];
        int lines = 0;
        if (q0 < 0 || q1 < q0 || (int64_t)q1 > a.n_seq) {
            flag(a.status, WH_STATUS_BAD_OFFSET);
            lines = -1;
        } else {
            for (int q = q0; q < q1; ++q) {
                const int o = a.order_seq[q];
                int lb, le;
                const int c = order_lines_checked(a, o, lb, le);
                if (c < 0) {
                    flag(a.status, WH_STATUS_BAD_ORDER);
                    lines = -1;
                    break;
                }
                lines += c;
                M.order_tour[(int64_t)p * a.n_orders + o] = t;
            }
        }
        M.tour_lines[t] = lines;
    }
}

// The same index built one plan per CTA (grid stride over plans): the
// plan's order -> tour row is filled in shared memory (-1 where the plan does
// not hold the order) and written out in one coalesced pass, so the table
// needs no clearing pass and no tour searches for its plan.  Used when a row
// fits MVT_MAX_ORDERS entries.
constexpr int MVT_THREADS = 256;
constexpr int MVT_MAX_ORDERS = 12288;   // 48 KB of shared memory

__global__ void __launch_bounds__(MVT_THREADS) k_mv_tours_plan(MoveArgs M) {
    extern __shared__ int32_t s_row[];
    const EvalArgs& a = M.a;
    for (int p = blockIdx.x; p < a.n_plans; p += gridDim.x) {
        for (int o = threadIdx.x; o < a.n_orders; o += blockDim.x) s_row[o] = -1;
        __syncthreads();
        int t0 = a.plan_tour_off[p], t1 = a.plan_tour_off[p + 1];
        if (t0 < 0 || t1 < t0 || t1 > a.n_tours || (p == 0 && t0 != 0) || (p == a.n_plans - 1 && t1 != a.n_tours)) {
            if (threadIdx.x == 0) flag(a.status, WH_STATUS_BAD_OFFSET);
            t0 = max(t0, 0);
            t1 = min(t1, a.n_tours);
        }
        for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
            const int q0 = a.tour_off[t], q1 = a.tour_off[t + 1];
            int lines = 0;
            if (q0 < 0 || q1 < q0 || (int64_t)q1 > a.n_seq) {
                flag(a.status, WH_STATUS_BAD_OFFSET);
                lines = -1;
            } else {
                for (int q = q0; q < q1; ++q) {
                    const int o = a.order_seq[q];
                    int lb, le;
                    const int c = order_lines_checked(a, o, lb, le);
                    if (c < 0) {
                        flag(a.status, WH_STATUS_BAD_ORDER);
                        lines = -1;
                        break;
                    }
                    lines += c;
                    s_row[o] = t;
                }
            }
            M.tour_lines[t] = lines;
        }
        __syncthreads();
        int32_t* row = M.order_tour + (int64_t)p * a.n_orders;
        for (int o = threadIdx.x; o < a.n_orders; o += blockDim.x) row[o] = s_row[o];
        __syncthreads();
    }
}

__global__ void k_mv_sku_count(MoveArgs M) {
    const EvalArgs& a = M.a;
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < a.n_lines; l += gridDim.x * blockDim.x) {
        const int s = a.line_sku[l];
        if ((unsigned)s < (unsigned)a.n_sku) atomicAdd(&M.sku_cur[s], 1);
    }
}

// one block: exclusive scan of the per-SKU counts into sku_off, cursors reset
__global__ void k_mv_sku_scan(MoveArgs M) {
    __shared__ int warp_tot[32];
    __shared__ int carry;
    const int n = M.a.n_sku, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += blockDim.x) {
        const int i = base + tid;
        const int v = i < n ? M.sku_cur[i] : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += u;
        }
        if (lane == 31) warp_tot[w] = x;
        __syncthreads();
        if (w == 0) {
            int y = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, y, o);
                if (lane >= o) y += u;
            }
            warp_tot[lane] = y;
        }
        __syncthreads();
        const int excl = carry + (w ? warp_tot[w - 1] : 0) + x - v;
        if (i < n) {
            M.sku_off[i] = excl;
            M.sku_cur[i] = 0;
        }
        __syncthreads();
        if (tid == blockDim.x - 1) carry = excl + v;
        __syncthreads();
    }
    if (tid == 0) M.sku_off[n] = carry;
}

__global__ void k_mv_sku_fill(MoveArgs M) {
    const EvalArgs& a = M.a;
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < a.n_orders; o += gridDim.x * blockDim.x) {
        int lb, le;
        if (order_lines_checked(a, o, lb, le) < 0) continue;
        for (int l = lb; l < le; ++l) {
            const int s = a.line_sku[l];
            if ((unsigned)s >= (unsigned)a.n_sku) continue;
            const int k = atomicAdd(&M.sku_cur[s], 1);
            M.sku_orders[M.sku_off[s] + k] = o;
        }
    }
}

// status and task count of every move; deltas zeroed
__global__ void k_mv_count(MoveArgs M) {
    const EvalArgs& a = M.a;
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < M.n_moves; m += gridDim.x * blockDim.x) {
        const int4 mv = M.moves[m];
        M.delta[2 * m] = 0;
        M.delta[2 * m + 1] = 0;
        int st = 3, cnt = 0;
        const int p = mv.w;
        if (p >= 0 && p < a.n_plans) {
            const int64_t row = (int64_t)p * a.n_orders;
            if (mv.x == 0 || mv.x == 1) {
                int lb, le;
                const int la = order_lines_checked(a, mv.y, lb, le);
                const int ta = la >= 0 ? M.order_tour[row + mv.y] : -1;
                if (ta >= 0 && M.tour_lines[ta] >= 0) {
                    if (mv.x == 0) {
                        const int lbb = order_lines_checked(a, mv.z, lb, le);
                        const int tb = lbb >= 0 ? M.order_tour[row + mv.z] : -1;
                        if (tb >= 0 && M.tour_lines[tb] >= 0) {
                            if (ta == tb) st = 2;
                            else if (M.max_lines > 0 && (M.tour_lines[ta] - la + lbb > M.max_lines ||
                                                         M.tour_lines[tb] - lbb + la > M.max_lines)) st = 1;
                            else { st = 0; cnt = 2; }
                        }
                    } else {
                        const int n_t = a.plan_tour_off[p + 1] - a.plan_tour_off[p];
                        if (mv.z >= 0 && mv.z < n_t) {
                            const int tb = a.plan_tour_off[p] + mv.z;
                            if (tb == ta) st = 2;
                            else if (M.tour_lines[tb] < 0) st = 3;
                            else if ((M.max_orders > 0 && a.tour_off[tb + 1] - a.tour_off[tb] + 1 > M.max_orders) ||
                                     (M.max_lines > 0 && M.tour_lines[tb] + la > M.max_lines)) st = 1;
                            else { st = 0; cnt = 2; }
                        }
                    }
                }
            } else if (mv.x == 2) {
                if (a.slot_stride > 0 && (unsigned)mv.y < (unsigned)a.n_sku && (unsigned)mv.z < (unsigned)a.n_sku) {
                    if (mv.y == mv.z) st = 2;
                    else {
                        st = 0;
                        cnt = (M.sku_off[mv.y + 1] - M.sku_off[mv.y]) + (M.sku_off[mv.z + 1] - M.sku_off[mv.z]);
                    }
                }
            } else if (mv.x == 3) {
                // relocation of SKU mv.y to location mv.z, which must be empty
                if (a.slot_stride > 0 && a.loc_used && (unsigned)mv.y < (unsigned)a.n_sku &&
                    (unsigned)mv.z < (unsigned)a.g.n_loc) {
                    const int words = (a.g.n_loc + 31) >> 5;
                    const uint32_t used = a.loc_used[(int64_t)p * words + (mv.z >> 5)] >> (mv.z & 31) & 1u;
                    if (a.slot_map[(int64_t)p * a.slot_stride + mv.y] == mv.z) st = 2;
                    else if (!used) {
                        st = 0;
                        cnt = M.sku_off[mv.y + 1] - M.sku_off[mv.y];
                    }
                }
            }
        }
        M.mstatus[m] = st;
        M.task_off[m] = cnt;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        M.task_off[M.n_moves] = 0;
        *M.long_count = 0;
        if (M.stats) M.stats[0] = M.stats[1] = 0;
    }
}

// ---- exclusive scan of int64 counts in place (n+1 entries): block scans,
// a scan of the block totals, then the carries added
constexpr int SCAN_T = 1024;

__device__ __forceinline__ long long block_excl_scan(long long v, long long* warp_tot, long long& total) {
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long u = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += u;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        long long y = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long u = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += u;
        }
        warp_tot[lane] = y;
    }
    __syncthreads();
    total = warp_tot[(blockDim.x >> 5) - 1];
    const long long r = (w ? warp_tot[w - 1] : 0) + x - v;
    __syncthreads();
    return r;
}

__global__ void k_scan_blocks(int64_t* v, int64_t n, int64_t* block_tot) {
    __shared__ long long wt[32];
    const int64_t i = (int64_t)blockIdx.x * SCAN_T + threadIdx.x;
    const long long x = i < n ? v[i] : 0;
    long long tot;
    const long long e = block_excl_scan(x, wt, tot);
    if (i < n) v[i] = e;
    if (threadIdx.x == 0) block_tot[blockIdx.x] = tot;
}

__global__ void k_scan_top(int64_t* block_tot, int nb) {
    __shared__ long long wt[32];
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += SCAN_T) {
        const int i = base + threadIdx.x;
        const long long x = i < nb ? block_tot[i] : 0;
        long long tot;
        const long long e = block_excl_scan(x, wt, tot);
        const long long c = carry;
        if (i < nb) block_tot[i] = c + e;
        __syncthreads();
        if (threadIdx.x == 0) carry = c + tot;
        __syncthreads();
    }
}

__global__ void k_scan_add(int64_t* v, int64_t n, const int64_t* block_tot) {
    const int64_t i = (int64_t)blockIdx.x * SCAN_T + threadIdx.x;
    if (i < n) v[i] += block_tot[blockIdx.x];
}

// task = {move, tour, order, tag}: tag >= 0 or -1: order moves (tag = order
// removed, order = order added, -1 = none); tag -2 / -3: SKU swap, `order` is
// the order of s1's / s2's list the task came from.  One move per lane; a SKU
// list longer than MVF_SERIAL orders (a popular SKU can sit in hundreds) is
// written by the whole warp, 32 tasks a step, at the same places.
constexpr int MVF_SERIAL = 32;

__global__ void k_mv_fill(MoveArgs M) {
    const EvalArgs& a = M.a;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < M.n_moves; base += stride) {
        const int m = (int)(base + lane);
        int lb[2] = {0, 0}, ln[2] = {0, 0}, lk[2] = {0, 0};   // a long list per side: begin, length, first task
        int64_t row = 0, t0 = 0;
        if (m < M.n_moves && M.mstatus[m] == 0) {
            const int4 mv = M.moves[m];
            row = (int64_t)mv.w * a.n_orders;
            t0 = M.task_off[m];
            int4* out = M.tasks + t0;
            if (mv.x == 0) {
                const int ta = M.order_tour[row + mv.y], tb = M.order_tour[row + mv.z];
                out[0] = make_int4(m, ta, mv.z, mv.y);
                out[1] = make_int4(m, tb, mv.y, mv.z);
            } else if (mv.x == 1) {
                const int ta = M.order_tour[row + mv.y], tb = a.plan_tour_off[mv.w] + mv.z;
                out[0] = make_int4(m, ta, -1, mv.y);
                out[1] = make_int4(m, tb, mv.y, -1);
            } else {
                int k = 0;
                for (int side = 0; side < (mv.x == 2 ? 2 : 1); ++side) {
                    const int sk = side ? mv.z : mv.y;
                    const int b = M.sku_off[sk], e = M.sku_off[sk + 1];
                    if (e - b > MVF_SERIAL) {
                        lb[side] = b;
                        ln[side] = e - b;
                        lk[side] = k;
                        k += e - b;
                        continue;
                    }
                    for (int i = b; i < e; ++i) {
                        const int o = M.sku_orders[i];
                        out[k++] = make_int4(m, M.order_tour[row + o], o, side ? -3 : -2);
                    }
                }
            }
        }
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            unsigned longs = __ballot_sync(0xffffffffu, ln[side] > 0);
            while (longs) {
                const int src = __ffs(longs) - 1;
                longs &= longs - 1;
                const int b = __shfl_sync(0xffffffffu, lb[side], src), n = __shfl_sync(0xffffffffu, ln[side], src);
                const int k0 = __shfl_sync(0xffffffffu, lk[side], src), mm = __shfl_sync(0xffffffffu, m, src);
                const int64_t r = __shfl_sync(0xffffffffu, row, src);
                int4* out = M.tasks + __shfl_sync(0xffffffffu, t0, src) + k0;
                for (int i = lane; i < n; i += 32) {
                    const int o = M.sku_orders[b + i];
                    out[i] = make_int4(mm, M.order_tour[r + o], o, side ? -3 : -2);
                }
            }
        }
    }
}

// Location of SKU s under the move's slotting: the swapped pair for a SKU
// swap, the target location for the relocated SKU.
__device__ __forceinline__ int task_loc(const int32_t* map, int s, const int4 mv) {
    if (mv.x == 2) s = s == mv.y ? mv.z : (s == mv.z ? mv.y : s);
    else if (mv.x == 3 && s == mv.y) return mv.z;
    return map[s];
}

// the line's SKU is one the SKU move changes
__device__ __forceinline__ bool sku_hit(int s, const int4 mv) { return s == mv.y || (mv.x == 2 && s == mv.z); }

// Walk the changed tour of task `tk`: calls emit(key) for every line, in
// order; returns false on an invalid id.  For SKU-swap tasks also reports
// whether the task is the counted one of its tour.
template <typename Emit>
__device__ __forceinline__ bool walk_task(const MoveArgs& M, const int4 tk, const int4 mv, bool& primary,
                                          Emit emit) {
    const EvalArgs& a = M.a;
    const bool swap = mv.x >= 2;   // SKU moves: swap or relocation
    const int32_t* map = a.slot_map + (int64_t)mv.w * a.slot_stride;
    const int q0 = a.tour_off[tk.y], q1 = a.tour_off[tk.y + 1];
    const int add = (!swap && tk.z >= 0) ? tk.z : -1;
    const int rem = (!swap && tk.w >= 0) ? tk.w : -1;
    int hit_min = 0x7fffffff;
    bool own_has_s1 = false;
    bool ok = q0 >= 0 && q1 >= q0 && (int64_t)q1 <= a.n_seq;
    // the orders walked: positions q0..q1-1 of order_seq (without `rem`),
    // then the added order; ids two ahead and line bounds one ahead are in
    // flight while the current order's lines are gathered
    const int q_end = !ok ? q0 : (add >= 0 ? q1 + 1 : q1);
    auto order_at = [&](int q) { return q < q1 ? a.order_seq[q] : add; };
    int o0 = q0 < q_end ? order_at(q0) : 0;
    int o1 = q0 + 1 < q_end ? order_at(q0 + 1) : 0;
    int lb0 = 0, le0 = 0;
    bool v0 = q0 < q_end && order_lines_checked(a, o0, lb0, le0) >= 0;
    for (int q = q0; ok && q < q_end; ++q) {
        const int o = o0;
        const int lb = lb0, le = le0;
        const bool valid = v0;
        const int o2 = q + 2 < q_end ? order_at(q + 2) : 0;
        v0 = q + 1 < q_end && order_lines_checked(a, o1, lb0, le0) >= 0;
        o0 = o1;
        o1 = o2;
        if (q < q1 && o == rem) continue;
        if (!valid) { ok = false; break; }
        // four lines at a time: their SKU loads, then their slot loads (the
        // plan's own slotting, mostly DRAM), are in flight together
        for (int l = lb; ok && l < le; l += 4) {
            int sk[4], loc[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) sk[j] = l + j < le ? a.line_sku[l + j] : 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                loc[j] = -1;
                if (l + j >= le) continue;
                const int sj = sk[j];
                if ((unsigned)sj >= (unsigned)a.n_sku) { ok = false; continue; }
                if (swap && sku_hit(sj, mv)) {
                    hit_min = min(hit_min, o);
                    if (o == tk.z && sj == mv.y) own_has_s1 = true;
                }
                loc[j] = task_loc(map, sj, mv);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (!ok || l + j >= le) continue;
                if ((unsigned)loc[j] >= (unsigned)a.g.n_loc) { ok = false; continue; }
                emit(loc_key(a.g, loc[j]));
            }
        }
    }
    primary = !swap || (hit_min == tk.z && (tk.w == -2 || !own_has_s1));
    return ok;
}

template <bool KEY16>
__global__ void __launch_bounds__(MV_THREADS) k_mv_eval(MoveArgs M) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31;
    uint32_t* col16 = reinterpret_cast<uint32_t*>(smem) + tid;
    uint2* col32 = reinterpret_cast<uint2*>(smem) + tid;
    const EvalArgs& a = M.a;
    const int64_t n_tasks = M.n_tasks;
    const int64_t warps = (int64_t)gridDim.x * (T >> 5);
    for (int64_t base = ((int64_t)blockIdx.x * (T >> 5) + (tid >> 5)) * 32; base < n_tasks; base += warps * 32) {
        const int64_t i = base + lane;
        const bool active = i < n_tasks;
        int4 tk = make_int4(-1, -1, -1, -1), mv = make_int4(0, 0, 0, 0);
        int n = 0;
        bool ok = false, primary = false;
        if (active) {
            tk = M.tasks[i];
            mv = M.moves[tk.x];
            if (tk.y >= 0 && tk.y < a.n_tours) {
                ok = walk_task(M, tk, mv, primary, [&](uint32_t k) {
                    if (n < SHORT_MAX) {
                        if constexpr (KEY16) reinterpret_cast<uint16_t*>(col16 + (n >> 1) * T)[n & 1] = (uint16_t)key16_of(k);
                        else reinterpret_cast<uint32_t*>(col32 + (n >> 1) * T)[n & 1] = k;
                    }
                    ++n;
                });
            } else {
                primary = false;   // an order of the SKU lists outside the plan
                ok = true;
            }
            if (!ok) {
                flag(a.status, WH_STATUS_BAD_ORDER);
                M.mstatus[tk.x] = 3;
            }
        }
        if (M.stats) {   // changed tours walked and their lines (the moves' roofline)
            const unsigned walked = __reduce_add_sync(0xffffffffu, active && ok ? 1u : 0u);
            const unsigned lines = __reduce_add_sync(0xffffffffu, active && ok ? (unsigned)n : 0u);
            if (lane == 0 && walked) {
                atomicAdd(M.stats, (unsigned long long)walked);
                atomicAdd(M.stats + 1, (unsigned long long)lines);
            }
        }
        bool run = active && ok && primary;
        bool deferred = false;
        if (run && n > SHORT_MAX) {
            const int slot = atomicAdd(M.long_count, 1);
            if (slot < M.long_cap) { M.long_list[slot] = (int32_t)i; deferred = true; }
            else { flag(a.status, WH_STATUS_LONG_OVERFLOW); M.mstatus[tk.x] = 3; }
            run = false;
        }
        const int nr = run ? n : 0;
        const int nmax = __reduce_max_sync(0xffffffffu, nr);
        int cs = 0, cr = 0, m = 0;
        if constexpr (KEY16) {
            if (nmax <= 16) tour16<8>(a, col16, T, nr, true, cs, cr, m);
            else if (nmax <= 32) tour16<16>(a, col16, T, nr, true, cs, cr, m);
            else tour16<32>(a, col16, T, nr, true, cs, cr, m);
        } else {
            if (nmax <= 16) tour32<16>(a, col32, T, nr, true, cs, cr, m);
            else if (nmax <= 32) tour32<32>(a, col32, T, nr, true, cs, cr, m);
            else tour32<64>(a, col32, T, nr, true, cs, cr, m);
        }
        // more pick aisles than this thread's record slots: the long-task
        // pass scores the task
        if (run && m > a.max_rec) {
            const int slot = atomicAdd(M.long_count, 1);
            if (slot < M.long_cap) { M.long_list[slot] = (int32_t)i; deferred = true; }
            else { flag(a.status, WH_STATUS_LONG_OVERFLOW); M.mstatus[tk.x] = 3; }
            run = false;
        }
        long long ds = 0, dr = 0;
        if (run) {
            ds = (long long)cs - M.tour_s_old[tk.y];
            dr = (long long)cr - M.tour_rr_old[tk.y];
        }
        if (active && !deferred)   // deferred tasks: k_mv_long writes
            M.task_cost[i] = run ? make_int2(cs, cr) : make_int2(-1, -1);
        const int key = active ? tk.x : -1;
        const long long ss = segmented_sum(ds, key, lane);
        const long long sr = segmented_sum(dr, key, lane);
        const int prev_key = __shfl_up_sync(0xffffffffu, key, 1);
        if (active && (lane == 0 || prev_key != key) && (ss || sr)) {
            atomicAdd(reinterpret_cast<unsigned long long*>(&M.delta[2 * tk.x]), (unsigned long long)ss);
            atomicAdd(reinterpret_cast<unsigned long long*>(&M.delta[2 * tk.x + 1]), (unsigned long long)sr);
        }
    }
}

// Warp-parallel form of walk_task: lane j takes the changed tour's orders
// j, j + 32, ... (the added order last) and stores their line indices at
// positions given by a warp prefix sum of the order line counts; then the
// lanes turn positions x, x + 32, ... into keys.  Only the first `cap`
// positions are stored.  Returns ok and sets n and primary (all warp-uniform).
__device__ __forceinline__ bool walk_task_warp(const MoveArgs& M, const int4 tk, const int4 mv, uint32_t* kb,
                                               int cap, int lane, int& n_out, bool& primary) {
    const EvalArgs& a = M.a;
    const bool swap = mv.x >= 2;   // SKU moves: swap or relocation
    const int32_t* map = a.slot_map + (int64_t)mv.w * a.slot_stride;
    const int q0 = a.tour_off[tk.y], q1 = a.tour_off[tk.y + 1];
    const int add = (!swap && tk.z >= 0) ? tk.z : -1;
    const int rem = (!swap && tk.w >= 0) ? tk.w : -1;
    bool bad = !(q0 >= 0 && q1 >= q0 && (int64_t)q1 <= a.n_seq);
    const int q_end = bad ? q0 : (add >= 0 ? q1 + 1 : q1);
    int hit_min = 0x7fffffff, n = 0;
    bool own_has_s1 = false;
    // the lines' indices at their positions in the changed tour (lanes over
    // orders; shared stores only)
    for (int qb = q0; qb < q_end; qb += 32) {
        const int q = qb + lane;
        int o = -1, lb = 0, le = 0;
        if (!bad && q < q_end) {
            o = q < q1 ? a.order_seq[q] : add;
            if (q < q1 && o == rem) o = -1;
            else if (order_lines_checked(a, o, lb, le) < 0) { bad = true; lb = le = 0; }
        }
        const int cnt = le - lb;
        const int incl = warp_inclusive_scan(cnt);
        int pos = n + incl - cnt;
        for (int l = lb; l < le; ++l, ++pos)
            if (pos < cap) kb[pos] = (uint32_t)l;
        n += __shfl_sync(0xffffffffu, incl, 31);
    }
    bad = __any_sync(0xffffffffu, bad);
    __syncwarp();
    // keys: lanes over positions, four a lane with their SKU and slot loads in
    // flight together.  A line whose SKU the move changes finds its orders
    // among the tour's (a SKU move keeps every order of the tour)
    const int nn = bad ? 0 : min(n, cap);
    for (int x0 = 0; x0 < nn; x0 += 128) {
        int l[4], sk[4], loc[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int x = x0 + 32 * u + lane;
            l[u] = x < nn ? (int)kb[x] : -1;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) sk[u] = l[u] >= 0 ? a.line_sku[l[u]] : -1;
#pragma unroll
        for (int u = 0; u < 4; ++u)
            loc[u] = (l[u] >= 0 && (unsigned)sk[u] < (unsigned)a.n_sku) ? task_loc(map, sk[u], mv) : -1;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (l[u] < 0) continue;
            if ((unsigned)sk[u] >= (unsigned)a.n_sku || (unsigned)loc[u] >= (unsigned)a.g.n_loc) {
                bad = true;
                continue;
            }
            if (swap && sku_hit(sk[u], mv)) {
                for (int q = q0; q < q1; ++q) {
                    const int o = a.order_seq[q];
                    if ((unsigned)o >= (unsigned)a.n_orders) continue;
                    if (l[u] >= a.order_off[o] && l[u] < a.order_off[o + 1]) {
                        hit_min = min(hit_min, o);
                        if (o == tk.z && sk[u] == mv.y) own_has_s1 = true;
                    }
                }
            }
            kb[x0 + 32 * u + lane] = loc_key(a.g, loc[u]);
        }
    }
    const bool ok = !__any_sync(0xffffffffu, bad);
    hit_min = __reduce_min_sync(0xffffffffu, hit_min);
    own_has_s1 = __any_sync(0xffffffffu, own_has_s1);
    primary = !swap || (hit_min == tk.z && (tk.w == -2 || !own_has_s1));
    n_out = n;
    return ok;
}

// Tasks of more than SHORT_MAX lines, in two kernels.  k_mv_long_rec: one
// warp per task walks the changed tour (walk_task_warp), sorts its keys in
// shared memory and extracts the per-aisle records in parallel (a ballot
// numbers the aisle runs) into a column matrix in global memory; a task with
// more than MVL_RMAX records runs its scan and DP on one lane right away.
// k_mv_long_dp: one task per thread runs the DP over its records (coalesced
// column reads), so the DP, one step per visited aisle, keeps every lane busy.
__device__ __forceinline__ void mv_long_commit(const MoveArgs& M, int64_t i, int cs, int cr) {
    const int4 tk = M.tasks[i];
    M.task_cost[i] = make_int2(cs, cr);
    const long long ds = (long long)cs - M.tour_s_old[tk.y];
    const long long dr = (long long)cr - M.tour_rr_old[tk.y];
    atomicAdd(reinterpret_cast<unsigned long long*>(&M.delta[2 * tk.x]), (unsigned long long)ds);
    atomicAdd(reinterpret_cast<unsigned long long*>(&M.delta[2 * tk.x + 1]), (unsigned long long)dr);
}

__global__ void __launch_bounds__(LONG_WARPS * 32, 6) k_mv_long_rec(MoveArgs M) {
    __shared__ uint32_t buf[LONG_WARPS][LONG_MAXL];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int count = min(min(*M.long_count, M.long_cap), M.long_rec_cap);
    uint32_t* kb = buf[warp];
    const EvalArgs& a = M.a;
    const int64_t cap = M.long_rec_cap;
    for (int w = blockIdx.x * LONG_WARPS + warp; w < count; w += gridDim.x * LONG_WARPS) {
        const int64_t i = M.long_list[w];
        const int4 tk = M.tasks[i];
        const int4 mv = M.moves[tk.x];
        int n = 0;
        bool primary = false;
        const bool ok = walk_task_warp(M, tk, mv, kb, LONG_MAXL, lane, n, primary);
        __syncwarp();
        if (!ok || n > LONG_MAXL || n < 1) {
            if (lane == 0) {
                flag(a.status, n > LONG_MAXL ? WH_STATUS_TOUR_TOO_LONG : WH_STATUS_BAD_ORDER);
                M.mstatus[tk.x] = 3;
                M.task_cost[i] = make_int2(-1, -1);
                M.long_m[w] = -1;
            }
            __syncwarp();
            continue;
        }
        warp_sort_buffer(kb, n, lane);
        // per-aisle records: run r of the sorted keys -> long_rec[r * cap + w]
        int m = 0;
        for (int x0 = 0; x0 < n; x0 += 32) {
            const int x = x0 + lane;
            const bool in = x < n;
            const uint32_t key = in ? kb[x] : 0u;
            const int ai = (int)(key >> 16);
            const bool first = in && (x == 0 || (int)(kb[x - 1] >> 16) != ai);
            const bool last = in && (x == n - 1 || (int)(kb[x + 1] >> 16) != ai);
            const unsigned fm = __ballot_sync(0xffffffffu, first);
            const int r = m + __popc(fm & ((2u << lane) - 1u)) - 1;
            if (last && r < MVL_RMAX) {
                const int hi = (int)(key & 0xFFFFu);
                int lo = hi, gi = 0;
                for (int y = x; y > 0 && (int)(kb[y - 1] >> 16) == ai; --y) {
                    const int kp = (int)(kb[y - 1] & 0xFFFFu);
                    gi = max(gi, lo - kp);
                    lo = kp;
                }
                M.long_rec[r * cap + w] =
                    make_uint2(((uint32_t)ai << 16) | (uint32_t)lo, ((uint32_t)hi << 16) | (uint32_t)gi);
            }
            m += __popc(fm);
        }
        if (lane == 0) {
            const uint32_t kl = kb[n - 1];   // rightmost aisle, its deepest slot
            M.long_key[w] = kl;
            if (m <= MVL_RMAX) {
                M.long_m[w] = m;
            } else {
                // more aisles than the record matrix keeps: scan and DP here
                M.long_m[w] = -1;
                DP5 v;
                dp_init(v);
                int pa = 0, lo = 0, prev = 0, gi = 0;
                for (int x = 0; x < n; ++x) {
                    const uint32_t key = kb[x];
                    const int ai = (int)(key >> 16), k = (int)(key & 0xFFFFu);
                    const bool first = (x == 0) || ((int)(kb[x - 1] >> 16) != ai);
                    const bool last = (x == n - 1) || ((int)(kb[x + 1] >> 16) != ai);
                    gi = first ? 0 : max(gi, k - prev);
                    lo = first ? k : lo;
                    prev = k;
                    if (last) {
                        dp_aisle(v, a.g, ai - pa, lo, k, gi);
                        pa = ai;
                    }
                }
                mv_long_commit(M, i, sshape_cost(a.g, m, (int)(kl >> 16), (int)(kl & 0xFFFFu)), dp_final(v));
            }
        }
        __syncwarp();
    }
}

__global__ void k_mv_long_dp(MoveArgs M) {
    const int count = min(min(*M.long_count, M.long_cap), M.long_rec_cap);
    for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < count; w += gridDim.x * blockDim.x) {
        const int m = M.long_m[w];
        if (m < 0) continue;
        const uint32_t kl = M.long_key[w];
        mv_long_commit(M, M.long_list[w], sshape_cost(M.a.g, m, (int)(kl >> 16), (int)(kl & 0xFFFFu)),
                       rr_records32_mem(M.a.g, M.long_rec + w, M.long_rec_cap, m));
    }
}

// moves that ended with a non-zero status report zero deltas
__global__ void k_mv_finish(MoveArgs M) {
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < M.n_moves; m += gridDim.x * blockDim.x) {
        if (M.mstatus[m] != 0) {
            M.delta[2 * m] = 0;
            M.delta[2 * m + 1] = 0;
        }
    }
}

int grid_of(int64_t n, int threads, int cap = 8192) {
    int64_t g = (n + threads - 1) / threads;
    if (g > cap) g = cap;
    return g < 1 ? 1 : (int)g;
}

// occupancy bits of every plan's slotting (relocation moves): bit l of plan
// p set when a SKU of p sits at location l (ids outside the layout skipped)
__global__ void k_occupancy(const int32_t* slot_map, int64_t stride, int32_t n_plans, int32_t n_sku, int32_t n_loc,
                            uint32_t* used) {
    const int64_t total = (int64_t)n_plans * n_sku;
    const int words = (n_loc + 31) >> 5;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = i / n_sku, s = i - p * n_sku;
        const int loc = slot_map[p * stride + s];
        if ((unsigned)loc < (unsigned)n_loc) atomicOr(&used[p * words + (loc >> 5)], 1u << (loc & 31));
    }
}

}  // namespace

cudaError_t launch_moves_prepare(const MoveArgs& M, int num_sms, cudaStream_t s, bool reuse_index) {
    const EvalArgs& a = M.a;
    if (reuse_index) {
        // the order -> tour table, the tours' line counts and the SKU ->
        // orders index of the same plans are in place: only the moves' checks,
        // task counts and their scan
        k_mv_count<<<grid_of(M.n_moves, 256), 256, 0, s>>>(M);
        const int64_t n = (int64_t)M.n_moves + 1;
        const int nb = (int)((n + SCAN_T - 1) / SCAN_T);
        k_scan_blocks<<<nb, SCAN_T, 0, s>>>(M.task_off, n, M.scan_aux);
        k_scan_top<<<1, SCAN_T, 0, s>>>(M.scan_aux, nb);
        k_scan_add<<<nb, SCAN_T, 0, s>>>(M.task_off, n, M.scan_aux);
        return cudaGetLastError();
    }
    const bool per_plan = a.n_orders <= MVT_MAX_ORDERS;
    if (!per_plan &&
        cudaMemsetAsync(M.order_tour, 0xFF, sizeof(int32_t) * (size_t)a.n_plans * (size_t)a.n_orders, s) != cudaSuccess)
        return cudaGetLastError();
    if (cudaMemsetAsync(M.sku_cur, 0, sizeof(int32_t) * ((size_t)a.n_sku + 1), s) != cudaSuccess)
        return cudaGetLastError();
    if (per_plan) {
        // tours outside every plan's range (malformed plan offsets, flagged)
        // keep the "bad tour" line count
        if (a.n_tours > 0 && cudaMemsetAsync(M.tour_lines, 0xFF, sizeof(int32_t) * (size_t)a.n_tours, s) != cudaSuccess)
            return cudaGetLastError();
        const int grid = a.n_plans < num_sms * 8 ? a.n_plans : num_sms * 8;
        if (grid > 0) k_mv_tours_plan<<<grid, MVT_THREADS, sizeof(int32_t) * (size_t)a.n_orders, s>>>(M);
    } else if (a.n_tours > 0) {
        k_mv_tours<<<grid_of(a.n_tours, 256), 256, 0, s>>>(M);
    }
    if (a.n_lines > 0) k_mv_sku_count<<<grid_of(a.n_lines, 256), 256, 0, s>>>(M);
    k_mv_sku_scan<<<1, 1024, 0, s>>>(M);
    if (a.n_orders > 0) k_mv_sku_fill<<<grid_of(a.n_orders, 256), 256, 0, s>>>(M);
    k_mv_count<<<grid_of(M.n_moves, 256), 256, 0, s>>>(M);
    // exclusive scan of n_moves + 1 task counts
    const int64_t n = (int64_t)M.n_moves + 1;
    const int nb = (int)((n + SCAN_T - 1) / SCAN_T);
    k_scan_blocks<<<nb, SCAN_T, 0, s>>>(M.task_off, n, M.scan_aux);
    k_scan_top<<<1, SCAN_T, 0, s>>>(M.scan_aux, nb);
    k_scan_add<<<nb, SCAN_T, 0, s>>>(M.task_off, n, M.scan_aux);
    return cudaGetLastError();
}

size_t moves_eval_smem_bytes(bool k16, int max_rec) {
    const size_t slots = max_rec > SHORT_MAX / 2 ? (size_t)max_rec : (size_t)(SHORT_MAX / 2);
    return (k16 ? sizeof(uint32_t) : sizeof(uint2)) * slots * MV_THREADS;
}

cudaError_t launch_moves_fill(const MoveArgs& M, cudaStream_t s) {
    if (M.n_moves > 0) k_mv_fill<<<grid_of(M.n_moves, 256), 256, 0, s>>>(M);
    return cudaGetLastError();
}

cudaError_t launch_moves_eval(const MoveArgs& M, bool k16, int num_sms, cudaStream_t s) {
    if (M.n_moves > 0) k_mv_fill<<<grid_of(M.n_moves, 256), 256, 0, s>>>(M);
    if (M.n_tasks > 0) {
        const size_t smem = moves_eval_smem_bytes(k16, M.a.max_rec);
        auto kern = k16 ? k_mv_eval<true> : k_mv_eval<false>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, MV_THREADS, smem);
        if (e != cudaSuccess) return e;
        int64_t want = (M.n_tasks + MV_THREADS - 1) / MV_THREADS;
        int grid = per_sm * num_sms;
        if (grid > want) grid = (int)want;
        if (grid < 1) grid = 1;
        kern<<<grid, MV_THREADS, smem, s>>>(M);
    }
    return cudaGetLastError();
}

cudaError_t launch_moves_long(const MoveArgs& M, int num_sms, cudaStream_t s) {
    if (M.n_tasks > 0 && M.long_rec_cap > 0) {
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mv_long_rec, LONG_WARPS * 32, 0);
        if (e != cudaSuccess) return e;
        k_mv_long_rec<<<num_sms * (per_sm > 0 ? per_sm : 1), LONG_WARPS * 32, 0, s>>>(M);
        k_mv_long_dp<<<grid_of(M.long_rec_cap, 128), 128, 0, s>>>(M);
    }
    if (M.n_moves > 0) k_mv_finish<<<grid_of(M.n_moves, 256), 256, 0, s>>>(M);
    return cudaGetLastError();
}

}  // namespace wh

// ---------------------------------------------------------- local search
namespace wh {
namespace {

// One CTA per plan: the move with the most negative optimal-cost delta among
// the plan's moves of status 0 (ties: lowest index) is applied in place.
__global__ void k_ls_apply(LsArgs L) {
    extern __shared__ int32_t seg[];
    __shared__ long long s_best;
    __shared__ int s_pos[2];
    const EvalArgs& a = L.a;
    const int tid = threadIdx.x, T = blockDim.x;
    for (int p = blockIdx.x; p < a.n_plans; p += gridDim.x) {
        if (tid < 32) {
            long long best = 0x7fffffffffffffffll;
            for (int k = tid; k < L.moves_per_plan; k += 32) {
                const int64_t m = (int64_t)p * L.moves_per_plan + k;
                const long long d = L.delta[2 * m + 1];
                if (L.status[m] == 0 && d < 0 && L.moves[m].w == p) best = min(best, d * 256 + k);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
            if (tid == 0) {
                s_best = best;
                s_pos[0] = s_pos[1] = -1;
            }
        }
        __syncthreads();
        const long long best = s_best;
        const int k = best == 0x7fffffffffffffffll ? -1 : (int)(((best % 256) + 256) % 256);
        if (tid == 0) L.applied[p] = k;
        if (k >= 0) {
            const int4 mv = L.moves[(int64_t)p * L.moves_per_plan + k];
            const int t0 = a.plan_tour_off[p], t1 = a.plan_tour_off[p + 1];
            const int s0 = a.tour_off[t0], s1 = a.tour_off[t1];
            int32_t* order_seq = const_cast<int32_t*>(a.order_seq);
            int32_t* tour_off = const_cast<int32_t*>(a.tour_off);
            if (mv.x == 0 || mv.x == 1) {
                for (int q = s0 + tid; q < s1; q += T) {
                    const int o = order_seq[q];
                    if (o == mv.y) s_pos[0] = q;
                    if (mv.x == 0 && o == mv.z) s_pos[1] = q;
                }
                __syncthreads();
                const int ia = s_pos[0];
                if (mv.x == 0) {
                    if (tid == 0 && ia >= 0 && s_pos[1] >= 0) {
                        order_seq[ia] = mv.z;
                        order_seq[s_pos[1]] = mv.y;
                    }
                } else if (ia >= 0) {
                    // tour holding position ia: largest t with tour_off[t] <= ia
                    int lo = t0, hi = t1 - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (tour_off[mid] <= ia) lo = mid; else hi = mid - 1;
                    }
                    const int ta = lo, tb = t0 + mv.z;
                    const int end = tour_off[tb + 1];
                    const int r0 = tb > ta ? ia : end, r1 = tb > ta ? end : ia + 1;   // range that moves
                    if (r1 - r0 <= L.seg_cap) {
                        for (int q = r0 + tid; q < r1; q += T) seg[q - r0] = order_seq[q];
                        __syncthreads();
                        if (tb > ta) {
                            for (int q = r0 + tid; q < r1 - 1; q += T) order_seq[q] = seg[q - r0 + 1];
                            if (tid == 0) order_seq[r1 - 1] = mv.y;
                            for (int t = ta + 1 + tid; t <= tb; t += T) tour_off[t] -= 1;
                        } else {
                            for (int q = r0 + 1 + tid; q < r1; q += T) order_seq[q] = seg[q - r0 - 1];
                            if (tid == 0) order_seq[r0] = mv.y;
                            for (int t = tb + 1 + tid; t <= ta; t += T) tour_off[t] += 1;
                        }
                    } else if (tid == 0) {
                        flag(a.status, WH_STATUS_BAD_OFFSET);
                        L.applied[p] = -1;
                    }
                }
            } else if (mv.x == 2 && tid == 0) {
                int32_t* smap = const_cast<int32_t*>(a.slot_map) + (int64_t)p * a.slot_stride;
                const int32_t x = smap[mv.y];
                smap[mv.y] = smap[mv.z];
                smap[mv.z] = x;
            } else if (mv.x == 3 && tid == 0) {
                // relocation: the SKU's entry and the plan's occupancy bits
                int32_t* smap = const_cast<int32_t*>(a.slot_map) + (int64_t)p * a.slot_stride;
                const int32_t old = smap[mv.y];
                smap[mv.y] = mv.z;
                if (a.loc_used) {
                    uint32_t* used = a.loc_used + (int64_t)p * ((a.g.n_loc + 31) >> 5);
                    if ((unsigned)old < (unsigned)a.g.n_loc) used[old >> 5] &= ~(1u << (old & 31));
                    used[mv.z >> 5] |= 1u << (mv.z & 31);
                }
            }
            // costs: the changed tours take their tasks' new costs, the plan its delta
            if (L.task_cost && L.applied[p] == k) {
                const int64_t m = (int64_t)p * L.moves_per_plan + k;
                for (int64_t i = L.task_off[m] + tid; i < L.task_off[m + 1]; i += T) {
                    const int2 c = L.task_cost[i];
                    if (c.x < 0) continue;
                    const int t = L.tasks[i].y;
                    if (L.tour_s) L.tour_s[t] = c.x;
                    if (L.tour_rr) L.tour_rr[t] = c.y;
                    if (L.tour_changed) L.tour_changed[t] = 1;
                }
                if (tid == 0) {
                    if (L.plan_s) L.plan_s[p] += L.delta[2 * m];
                    if (L.plan_rr) L.plan_rr[p] += L.delta[2 * m + 1];
                }
            }
        }
        __syncthreads();
    }
}

// Features of every task's changed tour, one task per warp (WarpFeat): the
// same walk as walk_task with lane j taking the tour's orders j, j + 32, ...
// (the added order last); the SKU-swap rule that picks the counted task of
// a tour reduces over the lanes.  Marks in task_cost which tasks count
// (rows of non-counted tasks are written too and ignored by the selection).
constexpr int TF_THREADS = 256;

// One changed tour per warp.  Its orders are taken 32 at a time (one per
// lane: id, line range); then the lanes walk the round's lines flat, 32 at a
// time, each lane finding its line's order from the orders' start offsets (a
// bitmask of order starts within the 32-line window), so all lanes gather
// slot-map entries together whatever the orders' sizes.
__global__ void __launch_bounds__(TF_THREADS) k_task_features(MoveArgs M, FeatConst c, uint4* X) {
    __shared__ WarpFeat ws[TF_THREADS / 32];
    __shared__ int s_lb[TF_THREADS / 32][32], s_off[TF_THREADS / 32][33], s_o[TF_THREADS / 32][32],
        s_rank[TF_THREADS / 32][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    WarpFeat& w = ws[wid];
    int* lbs = s_lb[wid];
    int* offs = s_off[wid];
    int* ords = s_o[wid];
    int* rank_to_k = s_rank[wid];
    wf_init(w, lane);
    const EvalArgs& a = M.a;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int64_t n_warps = (int64_t)gridDim.x * (TF_THREADS / 32);
    for (int64_t i = (int64_t)blockIdx.x * (TF_THREADS / 32) + wid; i < M.n_tasks; i += n_warps) {
        const int4 tk = M.tasks[i];
        bool ok = false, primary = false, over = false;
        uint32_t n_lines = 0;
        if (tk.y >= 0 && tk.y < a.n_tours) {
            const int4 mv = M.moves[tk.x];
            const bool swap = mv.x >= 2;   // SKU moves: swap or relocation
            const int32_t* map = a.slot_map + (int64_t)mv.w * a.slot_stride;
            const int q0 = a.tour_off[tk.y], q1 = a.tour_off[tk.y + 1];
            const int add = (!swap && tk.z >= 0) ? tk.z : -1;
            const int rem = (!swap && tk.w >= 0) ? tk.w : -1;
            bool bad = !(q0 >= 0 && q1 >= q0 && (int64_t)q1 <= a.n_seq);
            int hit_min = 0x7fffffff;
            bool own_has_s1 = false;
            const int q_end = bad ? q0 : (add >= 0 ? q1 + 1 : q1);
            for (int qb = q0; qb < q_end; qb += 32) {
                // this round's orders, one per lane (none: count 0)
                const int q = qb + lane;
                int o = -1, lb = 0, cnt = 0;
                if (q < q_end) {
                    o = q < q1 ? a.order_seq[q] : add;
                    if (q < q1 && o == rem) {
                        o = -1;
                    } else {
                        int le;
                        const int cc = order_lines_checked(a, o, lb, le);
                        if (cc < 0) bad = true;
                        else cnt = cc;
                    }
                }
                const int incl = warp_inclusive_scan(cnt);
                const int total = __shfl_sync(0xffffffffu, incl, 31);
                const unsigned nonempty = __ballot_sync(0xffffffffu, cnt > 0);
                lbs[lane] = lb;
                offs[lane] = incl - cnt;
                ords[lane] = o;
                if (cnt > 0) rank_to_k[__popc(nonempty & lt_mask)] = lane;
                __syncwarp();
                // the round's lines, 32 at a time: line p belongs to the
                // nonempty order whose start is the last one <= p
                int before = 0;   // nonempty orders starting before this window
                for (int p0 = 0; p0 < total; p0 += 32) {
                    const int start = offs[lane];
                    const bool head = cnt > 0 && start >= p0 && start < p0 + 32;
                    const unsigned hm = __reduce_or_sync(0xffffffffu, head ? 1u << (start - p0) : 0u);
                    const int p = p0 + lane;
                    if (p < total && !bad) {
                        const int r = before + __popc(hm & (lt_mask | (1u << lane))) - 1;
                        const int k = rank_to_k[r];
                        const int ok_ = ords[k];
                        const int l = lbs[k] + (p - offs[k]);
                        const int sk = a.line_sku[l];
                        if ((unsigned)sk >= (unsigned)a.n_sku) {
                            bad = true;
                        } else {
                            if (swap && sku_hit(sk, mv)) {
                                hit_min = min(hit_min, ok_);
                                if (ok_ == tk.z && sk == mv.y) own_has_s1 = true;
                            }
                            const int loc = task_loc(map, sk, mv);
                            if ((unsigned)loc >= (unsigned)a.g.n_loc) bad = true;
                            else {
                                over |= !wf_insert(w, loc_key(a.g, loc));
                                ++n_lines;
                            }
                        }
                    }
                    before += __popc(hm);
                }
                __syncwarp();
            }
            ok = !__any_sync(0xffffffffu, bad);
            hit_min = __reduce_min_sync(0xffffffffu, hit_min);
            own_has_s1 = __any_sync(0xffffffffu, own_has_s1);
            primary = !swap || (hit_min == tk.z && (tk.w == -2 || !own_has_s1));
        }
        over = __any_sync(0xffffffffu, over);
        n_lines = __reduce_add_sync(0xffffffffu, n_lines);
        if (lane == 0) M.task_cost[i] = (ok && primary && !over) ? make_int2(0, 0) : make_int2(-1, -1);
        wf_finish(w, c, lane, n_lines, X + i * 24);
    }
}

// Predicted delta of every move (sum over its counted tasks, in order), then
// per plan the `keep` moves with the lowest predicted delta (ties: lowest
// index); unfilled places get an invalid move that scores status 3.
__global__ void k_screen_score(ScreenArgs S) {
    const MoveArgs& M = S.M;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // one move per lane; a move of more than MVF_SERIAL tasks is scored by the
    // whole warp: lanes load 32 tasks' terms at once, and every lane adds
    // them up in task order, so the sum is the serial one
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < M.n_moves; base += stride) {
        const int64_t m = base + lane;
        float sc = 3.0e38f;
        int64_t i0 = 0, i1 = 0;
        if (m < M.n_moves && M.mstatus[m] == 0) {
            sc = 0.0f;
            i0 = M.task_off[m];
            i1 = M.task_off[m + 1];
        }
        const bool lng = i1 - i0 > MVF_SERIAL;
        if (!lng)
            for (int64_t i = i0; i < i1; ++i) {
                const int4 tk = M.tasks[i];
                if (tk.y < 0) continue;
                // counted task: an order move, or the first task of its tour for a SKU swap
                const int2 c = M.task_cost[i];
                if (c.x < 0) continue;
                sc += S.y_task[i] - S.y_tour[tk.y];
            }
        unsigned longs = __ballot_sync(0xffffffffu, lng);
        while (longs) {
            const int src = __ffs(longs) - 1;
            longs &= longs - 1;
            const int64_t b = __shfl_sync(0xffffffffu, i0, src), e = __shfl_sync(0xffffffffu, i1, src);
            float acc = 0.0f;
            for (int64_t c0 = b; c0 < e; c0 += 32) {
                const int64_t i = c0 + lane;
                float term = 0.0f;
                bool counted = false;
                if (i < e) {
                    const int4 tk = M.tasks[i];
                    if (tk.y >= 0 && M.task_cost[i].x >= 0) {
                        counted = true;
                        term = S.y_task[i] - S.y_tour[tk.y];
                    }
                }
                const unsigned cm = __ballot_sync(0xffffffffu, counted);
                for (int j = 0; j < 32; ++j) {
                    const float tj = __shfl_sync(0xffffffffu, term, j);
                    if ((cm >> j) & 1u) acc += tj;
                }
            }
            if (lane == src) sc = acc;
        }
        if (m < M.n_moves) S.score[m] = sc;
    }
}

__global__ void k_screen_select(ScreenArgs S) {
    const int lane = threadIdx.x & 31;
    const int n_plans = S.M.a.n_plans;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); p < n_plans; p += warps) {
        uint32_t taken[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // up to 256 moves per plan
        for (int j = 0; j < S.keep; ++j) {
            float best = 3.0e38f;
            int bk = 0x7fffffff;
            for (int k = lane; k < S.moves_per_plan; k += 32) {
                if (taken[k >> 5] >> (k & 31) & 1u) continue;
                const float v = S.score[p * S.moves_per_plan + k];
                if (v < best || (v == best && k < bk)) { best = v; bk = k; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float ov = __shfl_xor_sync(0xffffffffu, best, o);
                const int ok = __shfl_xor_sync(0xffffffffu, bk, o);
                if (ov < best || (ov == best && ok < bk)) { best = ov; bk = ok; }
            }
            int4 out = make_int4(9, 0, 0, (int)p);
            if (best < 1.0e38f && bk < S.moves_per_plan) {
                out = S.M.moves[p * S.moves_per_plan + bk];
                taken[bk >> 5] |= 1u << (bk & 31);
            }
            if (lane == 0) S.kept[p * S.keep + j] = out;
        }
    }
}

}  // namespace

cudaError_t launch_task_features(const MoveArgs& M, const FeatConst& c, void* X, int num_sms, cudaStream_t s) {
    if (M.n_tasks == 0) return cudaSuccess;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_task_features, TF_THREADS, 0);
    if (e != cudaSuccess) return e;
    int64_t grid = (int64_t)per_sm * num_sms;
    const int64_t want = (M.n_tasks + TF_THREADS / 32 - 1) / (TF_THREADS / 32);
    if (grid > want) grid = want;
    if (grid < 1) grid = 1;
    k_task_features<<<(int)grid, TF_THREADS, 0, s>>>(M, c, static_cast<uint4*>(X));
    return cudaGetLastError();
}

cudaError_t launch_screen_select(const ScreenArgs& S, cudaStream_t s) {
    k_screen_score<<<grid_of(S.M.n_moves, 256), 256, 0, s>>>(S);
    k_screen_select<<<grid_of((int64_t)S.M.a.n_plans * 32, 256), 256, 0, s>>>(S);
    return cudaGetLastError();
}

cudaError_t launch_ls_apply(const LsArgs& L, cudaStream_t s) {
    const size_t smem = sizeof(int32_t) * (size_t)L.seg_cap;
    cudaError_t e = cudaFuncSetAttribute(k_ls_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int grid = L.a.n_plans < 65536 ? L.a.n_plans : 65536;
    if (grid < 1) grid = 1;
    k_ls_apply<<<grid, 256, smem, s>>>(L);
    return cudaGetLastError();
}

}  // namespace wh

namespace wh {
cudaError_t launch_occupancy(const int32_t* slot_map, int64_t stride, int32_t n_plans, int32_t n_sku, int32_t n_loc,
                             uint32_t* used, int num_sms, cudaStream_t st) {
    const size_t words = (size_t)((n_loc + 31) >> 5) * (size_t)n_plans;
    cudaError_t e = cudaMemsetAsync(used, 0, words * sizeof(uint32_t), st);
    if (e != cudaSuccess || n_plans == 0 || n_sku == 0) return e;
    const int64_t total = (int64_t)n_plans * n_sku;
    const int64_t want = (total + 255) / 256;
    const int grid = (int)(want < (int64_t)num_sms * 16 ? want : (int64_t)num_sms * 16);
    k_occupancy<<<grid, 256, 0, st>>>(slot_map, stride, n_plans, n_sku, n_loc, used);
    return cudaGetLastError();
}
}  // namespace wh
