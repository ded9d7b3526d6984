// Explicit optimal routes: for listed tours, the order in which a picker
// visits the tour's pick points along a shortest closed walk from the depot
// (the picking sequence the paper's case study asks for, Sec. 5 and Sec. 6),
// with its length.
//
// One tour per thread.  The tour's keys are gathered and sorted, the
// Ratliff-Rosenthal DP runs in the same reduced 5-class form as the
// evaluation kernels but records, per visited aisle and per new class, which
// arrival (source class and horizontal edge pattern over the aisle gaps) gave
// the minimum.  Backtracking from the cheapest final class fixes the route's
// subgraph: the horizontal edges between consecutive pick aisles (front,
// back: 0, 1 or 2 each) and every pick aisle's vertical option (traverse,
// double traverse, largest gap left out, from the front, from the back).  The
// subgraph has even degrees and one component; Hierholzer's algorithm walks
// it from the depot, and the picks are emitted in walking order: along a
// traversed aisle in the walking direction, on a spur (the out-and-back
// pieces of the gap, front and back options) when its end node is first
// reached.  The walk's length equals the DP's, so the emitted sequence, taken
// with shortest paths between consecutive points, is an optimal route.
#include "tour_core.cuh"

namespace wh {

namespace {

constexpr int RT_MAXL = ROUTE_MAX_POINTS;   // distinct pick points per tour
constexpr int RT_MAXM = RT_MAXL; // pick aisles per tour
constexpr int RT_MAXE = 6 * RT_MAXM;

// arrival codes: (source class, horizontal pattern front/back)
enum { H_UU11 = 0, H_E020 = 1, H_EE20 = 2, H_OE02 = 3, H_EE02 = 4, H_EE22 = 5, H_E222 = 6 };
// classes
enum { C_UU = 0, C_E0 = 1, C_OE = 2, C_EE = 3, C_E2 = 4 };
// vertical options
enum { V_T = 1, V_D = 2, V_G = 3, V_F = 4, V_B = 5 };

__device__ __forceinline__ int h_src(int h) {
    return h == H_UU11 ? C_UU : h == H_E020 ? C_E0 : h == H_OE02 ? C_OE : h == H_E222 ? C_E2 : C_EE;
}
__device__ __forceinline__ int h_front(int h) {
    return h == H_UU11 ? 1 : (h == H_E020 || h == H_EE20 || h == H_EE22 || h == H_E222) ? 2 : 0;
}
__device__ __forceinline__ int h_back(int h) {
    return h == H_UU11 ? 1 : (h == H_OE02 || h == H_EE02 || h == H_EE22 || h == H_E222) ? 2 : 0;
}
__device__ __forceinline__ int vert_of(int cls, int h) {
    switch (cls) {
        case C_UU: return h == H_UU11 ? V_G : V_T;
        case C_EE: return h == H_UU11 ? V_T : (h == H_EE22 ? V_G : V_D);
        case C_E0: return V_F;
        case C_OE: return V_B;
        default: return V_G;
    }
}

// first argmin over candidates (value, code)
__device__ __forceinline__ void take(int& best, int& code, int val, int c) {
    if (val < best) {
        best = val;
        code = c;
    }
}

// One pick aisle of the DP, the same values as dp_aisle; returns the arrival
// code of every new class (3 bits per class, class c at bits 3c..3c+2).
__device__ uint32_t dp_aisle_track(DP5& v, const Geo& g, int d, int lo, int hi, int gi) {
    const int h2 = 2 * g.P * d, h4 = h2 + h2;
    int hv[7];
    hv[H_UU11] = v.uu + h2;
    hv[H_E020] = v.e0 + h2;
    hv[H_EE20] = v.ee + h2;
    hv[H_OE02] = v.oe + h2;
    hv[H_EE02] = v.ee + h2;
    hv[H_EE22] = v.ee + h4;
    hv[H_E222] = v.e2 + h4;
    const int ylo = g.h + lo * g.S, yhi = g.h + hi * g.S;
    const int gap = max(max(ylo, gi * g.S), g.Y - yhi);
    const int cG = 2 * (g.Y - gap), cB = 2 * (g.Y - ylo), cF = 2 * yhi, cT = g.Y, cD = 2 * g.Y;
    const int big = 0x7fffffff;
    int uu = big, ee = big, e0 = big, oe = big, e2 = big;
    int kuu = 0, kee = 0, ke0 = 0, koe = 0, ke2 = 0;
    take(uu, kuu, hv[H_UU11] + cG, H_UU11);
    take(uu, kuu, hv[H_E020] + cT, H_E020);
    take(uu, kuu, hv[H_EE20] + cT, H_EE20);
    take(uu, kuu, hv[H_OE02] + cT, H_OE02);
    take(uu, kuu, hv[H_EE02] + cT, H_EE02);
    take(uu, kuu, hv[H_E222] + cT, H_E222);
    take(uu, kuu, hv[H_EE22] + cT, H_EE22);
    take(ee, kee, hv[H_UU11] + cT, H_UU11);
    take(ee, kee, hv[H_E020] + cD, H_E020);
    take(ee, kee, hv[H_EE20] + cD, H_EE20);
    take(ee, kee, hv[H_OE02] + cD, H_OE02);
    take(ee, kee, hv[H_EE02] + cD, H_EE02);
    take(ee, kee, hv[H_E222] + cD, H_E222);
    take(ee, kee, hv[H_EE22] + cG, H_EE22);
    take(e0, ke0, hv[H_E020] + cF, H_E020);
    take(e0, ke0, hv[H_EE20] + cF, H_EE20);
    take(oe, koe, hv[H_OE02] + cB, H_OE02);
    take(oe, koe, hv[H_EE02] + cB, H_EE02);
    take(e2, ke2, hv[H_E020] + cG, H_E020);
    take(e2, ke2, hv[H_EE20] + cG, H_EE20);
    take(e2, ke2, hv[H_OE02] + cG, H_OE02);
    take(e2, ke2, hv[H_EE02] + cG, H_EE02);
    take(e2, ke2, hv[H_E222] + cG, H_E222);
    v.uu = uu;
    v.ee = ee;
    v.e0 = e0;
    v.oe = oe;
    v.e2 = e2;
    return (uint32_t)kuu | ((uint32_t)ke0 << 3) | ((uint32_t)koe << 6) | ((uint32_t)kee << 9) | ((uint32_t)ke2 << 12);
}

__global__ void __launch_bounds__(64) k_routes(EvalArgs a, const int32_t* tours, int32_t n, int32_t max_points,
                                               int32_t* points, int32_t* n_points, int32_t* length) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Geo& g = a.g;
    int32_t* out = points + (int64_t)i * max_points;
    n_points[i] = -1;
    length[i] = -1;
    const int t = tours[i];
    if ((unsigned)t >= (unsigned)a.n_tours) {
        flag(a.status, WH_STATUS_BAD_OFFSET);
        return;
    }
    int plan = 0;
    if (a.slot_stride != 0) {
        int lo = 0, hi = a.n_plans - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.plan_tour_off[mid] <= t) lo = mid; else hi = mid - 1;
        }
        plan = lo;
    }
    const int32_t* map = a.slot_map + (int64_t)plan * a.slot_stride;
    // gather the tour's distinct pick points (aisle << 16 | slot), ascending,
    // by insertion
    uint32_t key[RT_MAXL];
    int np = 0;
    const int q0 = a.tour_off[t], q1 = a.tour_off[t + 1];
    if (q0 < 0 || q1 < q0 || (int64_t)q1 > a.n_seq) {
        flag(a.status, WH_STATUS_BAD_OFFSET);
        return;
    }
    for (int q = q0; q < q1; ++q) {
        const int o = a.order_seq[q];
        if ((unsigned)o >= (unsigned)a.n_orders) {
            flag(a.status, WH_STATUS_BAD_ORDER);
            return;
        }
        const int l0 = a.order_off[o], l1 = a.order_off[o + 1];
        if (l0 < 0 || l1 < l0 || l1 > a.n_lines) {
            flag(a.status, WH_STATUS_BAD_OFFSET);
            return;
        }
        for (int l = l0; l < l1; ++l) {
            const int s = a.line_sku[l];
            const int loc = (unsigned)s < (unsigned)a.n_sku ? map[s] : -1;
            if ((unsigned)loc >= (unsigned)g.n_loc) {
                flag(a.status, WH_STATUS_BAD_LOC);
                return;
            }
            const uint32_t k = loc_key(g, loc);
            int y = np;
            while (y > 0 && key[y - 1] > k) --y;
            if (y > 0 && key[y - 1] == k) continue;   // the point is already in the tour
            if (np == RT_MAXL) {
                flag(a.status, WH_STATUS_TOUR_TOO_LONG);
                return;
            }
            for (int z = np; z > y; --z) key[z] = key[z - 1];
            key[y] = k;
            ++np;
        }
    }
    if (np > max_points) {
        flag(a.status, WH_STATUS_TOUR_TOO_LONG);
        return;
    }
    if (np == 0) {
        n_points[i] = 0;
        length[i] = 0;
        return;
    }
    // aisle runs [beg, end) of the points, the DP with decisions
    uint16_t beg[RT_MAXM + 1];
    uint16_t dec[RT_MAXM];
    int m = 0;
    DP5 v;
    dp_init(v);
    int pa = 0;
    for (int x = 0; x < np;) {
        if (m == RT_MAXM) {
            flag(a.status, WH_STATUS_TOUR_TOO_LONG);
            return;
        }
        const int ai = (int)(key[x] >> 16);
        int y = x + 1, gi = 0;
        while (y < np && (int)(key[y] >> 16) == ai) {
            gi = max(gi, (int)(key[y] & 0xFFFFu) - (int)(key[y - 1] & 0xFFFFu));
            ++y;
        }
        beg[m] = (uint16_t)x;
        dec[m] = (uint16_t)dp_aisle_track(v, g, ai - pa, (int)(key[x] & 0xFFFFu), (int)(key[y - 1] & 0xFFFFu), gi);
        pa = ai;
        ++m;
        x = y;
    }
    beg[m] = (uint16_t)np;
    int cls = C_EE, best = v.ee;
    if (v.e0 < best) { best = v.e0; cls = C_E0; }
    if (v.oe < best) { best = v.oe; cls = C_OE; }
    // backtrack: per pick aisle j, the edges into it from the left (front,
    // back: 0..2 each) and its vertical option, packed as hf | hb << 2 | vo << 4
    uint8_t cfg[RT_MAXM];
    for (int j = m - 1; j >= 0; --j) {
        const int h = (dec[j] >> (3 * cls)) & 7;
        cfg[j] = (uint8_t)(h_front(h) | (h_back(h) << 2) | (vert_of(cls, h) << 4));
        cls = h_src(h);
    }
    if (cls != C_E0 || ((cfg[0] >> 2) & 3) != 0) {   // the walk starts at the depot, on the front
        flag(a.status, WH_STATUS_BAD_OFFSET);
        return;
    }
    // spurs of the gap / front / back options: the front spur covers points
    // [beg, fs_end), the back spur [bs_beg, end) of the aisle
    uint16_t fs_end[RT_MAXM], bs_beg[RT_MAXM];
    for (int j = 0; j < m; ++j) {
        const int b0 = beg[j], b1 = beg[j + 1], vo = cfg[j] >> 4;
        fs_end[j] = (uint16_t)b0;
        bs_beg[j] = (uint16_t)b1;
        if (vo == V_F) {
            fs_end[j] = (uint16_t)b1;
        } else if (vo == V_B) {
            bs_beg[j] = (uint16_t)b0;
        } else if (vo == V_G) {
            // leave out the largest of the front gap, the inner gaps and the
            // back gap (the DP's choice; ties give the same length)
            const int lo = (int)(key[b0] & 0xFFFFu), hi = (int)(key[b1 - 1] & 0xFFFFu);
            const int gfront = g.h + lo * g.S, gback = g.Y - (g.h + hi * g.S);
            int gin = 0, split = b0;   // largest inner gap: between points split - 1 and split
            for (int x = b0 + 1; x < b1; ++x) {
                const int dgap = ((int)(key[x] & 0xFFFFu) - (int)(key[x - 1] & 0xFFFFu)) * g.S;
                if (dgap > gin) { gin = dgap; split = x; }
            }
            if (gfront >= gin && gfront >= gback) {
                bs_beg[j] = (uint16_t)b0;          // everything from the back
            } else if (gback >= gin) {
                fs_end[j] = (uint16_t)b1;          // everything from the front
            } else {
                fs_end[j] = (uint16_t)split;
                bs_beg[j] = (uint16_t)split;
            }
        }
    }
    // The route's multigraph: node 0 = depot, 1 + 2j = front end of pick aisle
    // j, 2 + 2j = its back end.  Edge 6j + c: c = 0, 1 the copies of the front
    // edge into aisle j, c = 2, 3 the back edge, c = 4, 5 the aisle traversal.
    // Every node has at most six incident edge slots, found in O(1).
    uint8_t used[RT_MAXM];
    for (int j = 0; j < m; ++j) used[j] = 0;
    auto exists = [&](int j, int c) -> bool {
        const int f = cfg[j];
        const int nv = (f >> 4) == V_T ? 1 : (f >> 4) == V_D ? 2 : 0;
        const int cnt = c < 2 ? (f & 3) : c < 4 ? ((f >> 2) & 3) : nv;
        return (c & 1) < cnt && !((used[j] >> c) & 1);
    };
    // an unused edge at node u: its id, and the node at its other end (-1: none)
    auto next_edge = [&](int u, int& other) -> int {
        if (u == 0) {
            for (int c = 0; c < 2; ++c)
                if (exists(0, c)) { other = 1; return c; }
            return -1;
        }
        const int j = (u - 1) >> 1;
        const bool front = (u & 1) != 0;
        const int c0 = front ? 0 : 2;
        for (int c = c0; c < c0 + 2; ++c)
            if (exists(j, c)) { other = j == 0 ? 0 : u - 2; return 6 * j + c; }
        if (j + 1 < m)
            for (int c = c0; c < c0 + 2; ++c)
                if (exists(j + 1, c)) { other = u + 2; return 6 * (j + 1) + c; }
        for (int c = 4; c < 6; ++c)
            if (exists(j, c)) { other = front ? u + 1 : u - 1; return 6 * j + c; }
        return -1;
    };
    // Hierholzer from the depot.  Nodes are popped in the order of an Euler
    // circuit (the reverse of the usual output, itself a circuit from the
    // depot); consecutive pops p_k, p_k+1 are joined by the edge p_k was
    // pushed along.  Picks are emitted while walking it: along an aisle the
    // first time it is traversed, in the walking direction; a spur's points
    // the first time its end node is reached.
    int n_edges = 0;
    for (int j = 0; j < m; ++j) {
        const int f = cfg[j];
        n_edges += (f & 3) + ((f >> 2) & 3) + ((f >> 4) == V_T ? 1 : (f >> 4) == V_D ? 2 : 0);
    }
    uint16_t st_node[RT_MAXE + 1], st_edge[RT_MAXE + 1];
    uint8_t seen[2 * RT_MAXM + 1], crossed[RT_MAXM];
    for (int x = 0; x <= 2 * m; ++x) seen[x] = 0;
    for (int j = 0; j < m; ++j) crossed[j] = 0;
    int w = 0, n_pop = 0, prev = -1, prev_e = 0;
    auto visit = [&](int node) {
        if (node == 0 || seen[node]) return;
        seen[node] = 1;
        const int j = (node - 1) >> 1;
        if (node & 1) {   // front end: up to the gap
            for (int x = beg[j]; x < fs_end[j]; ++x) out[w++] = (int32_t)key[x];
        } else {          // back end: down to the gap
            for (int x = beg[j + 1] - 1; x >= bs_beg[j]; --x) out[w++] = (int32_t)key[x];
        }
    };
    int sp = 1;
    st_node[0] = 0;
    st_edge[0] = 0xFFFF;
    while (sp > 0) {
        const int u = st_node[sp - 1];
        int other = -1;
        const int e = next_edge(u, other);
        if (e >= 0) {
            used[e / 6] |= (uint8_t)(1u << (e % 6));
            st_node[sp] = (uint16_t)other;
            st_edge[sp] = (uint16_t)e;
            ++sp;
            continue;
        }
        --sp;
        const int x = st_node[sp];
        if (prev >= 0) {   // walk prev -> x along prev_e
            const int j = prev_e / 6;
            if (prev_e % 6 >= 4 && !crossed[j]) {
                crossed[j] = 1;
                if (prev < x) {   // front -> back: deeper picks later
                    for (int y = beg[j]; y < beg[j + 1]; ++y) out[w++] = (int32_t)key[y];
                } else {
                    for (int y = beg[j + 1] - 1; y >= beg[j]; --y) out[w++] = (int32_t)key[y];
                }
            }
        }
        visit(x);
        prev = x;
        prev_e = st_edge[sp];
        ++n_pop;
    }
    if (n_pop != n_edges + 1 || prev != 0 || w != np) {
        flag(a.status, WH_STATUS_BAD_OFFSET);
        return;
    }
    n_points[i] = np;
    length[i] = dp_final(v);
}

}  // namespace

cudaError_t launch_routes(const EvalArgs& a, const int32_t* tours, int32_t n, int32_t max_points, int32_t* points,
                          int32_t* n_points, int32_t* length, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_routes<<<(n + 63) / 64, 64, 0, s>>>(a, tours, n, max_points, points, n_points, length);
    return cudaGetLastError();
}

}  // namespace wh
