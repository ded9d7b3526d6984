// Seed-and-grow batch formation on the GPU: the orders are partitioned into
// picker tours by the exact optimal route length (the paper's clustering of
// orders and suggestion of which orders are picked together, Sec. 5 and
// Sec. 6).  One CTA per slotting runs the greedy:
//   seed - the unassigned order whose tour alone is longest (ties: lowest id);
//   grow - add the fitting unassigned order that lengthens the tour least
//          (ties: lowest id) until the order or line capacity is reached or
//          no order fits;
// until every order is in a tour.
//
// The current tour lives in shared memory as one 256-bit pick-depth mask per
// aisle plus a per-aisle record (shallowest, deepest, largest gap between
// consecutive picks) and the sorted list of its aisles.  A candidate's length
// is the 5-class optimal-route DP over the union of the tour's aisles and the
// candidate's (merged in aisle order; the aisles the candidate touches take
// their record from the merged mask).  Each thread scores a strided share of
// the candidates; a block reduction on (increase << 32 | order id) picks the
// order, so ties resolve to the lowest id exactly as in the definition.
#include "tour_core.cuh"

namespace wh {

namespace {

constexpr int BG_THREADS = 256;

struct BgShared {
    uint16_t* key;       // [n_lines] aisle << 8 | slot under this slotting
    int32_t* off;        // [n_orders + 1]
    int32_t* alone;      // [n_orders] length of the order's tour alone
    uint32_t* mask;      // [A][8] the tour's pick-depth bits per aisle
    uint32_t* rec;       // [A] lo << 16 | hi << 8 | gap of the tour's aisles
    uint16_t* alist;     // [A] the tour's aisles, ascending
    int* n_aisles;       // entries of alist
    uint16_t* rem;       // [n_orders] the unassigned orders, compacted (any order)
    uint16_t* pos;       // [n_orders] position of an unassigned order in rem
};

// shallowest / deepest set slot and the largest gap between consecutive set
// slots of a 256-bit mask (at least one bit set)
__device__ __forceinline__ void mask_stats(const uint32_t (&m)[8], int& lo, int& hi, int& gap) {
    lo = -1;
    hi = -1;
    gap = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        uint32_t b = m[w];
        while (b) {
            const int k = 32 * w + __ffs(b) - 1;
            b &= b - 1;
            if (lo < 0) lo = k;
            else gap = max(gap, k - hi);
            hi = k;
        }
    }
}

// Optimal length of the tour plus order o (o < 0: the tour alone; with an
// empty tour: o alone).  The order's keys are sorted in S.key (setup).
__device__ int cost_with(const BgShared& S, const Geo& g, int o) {
    int io = 0, le = 0;
    if (o >= 0) {
        io = S.off[o];
        le = S.off[o + 1];
    }
    const bool has_o = io < le;
    const int nt = *S.n_aisles;
    DP5 v;
    dp_init(v);
    int pa = 0, it = 0;
    while (it < nt || io < le) {
        const int at = it < nt ? (int)S.alist[it] : 0x7fffffff;
        const int ao = io < le ? (int)(S.key[io] >> 8) : 0x7fffffff;
        const int a = min(at, ao);
        int lo, hi, gap;
        if (ao == a) {
            uint32_t m[8];
#pragma unroll
            for (int w = 0; w < 8; ++w) m[w] = at == a ? S.mask[a * 8 + w] : 0u;
            while (io < le && (int)(S.key[io] >> 8) == a) {
                const int k = S.key[io] & 0xFF;
                m[k >> 5] |= 1u << (k & 31);
                ++io;
            }
            mask_stats(m, lo, hi, gap);
            if (at == a) ++it;
        } else {
            const uint32_t r = S.rec[a];
            lo = (int)(r >> 16);
            hi = (int)((r >> 8) & 0xFF);
            gap = (int)(r & 0xFF);
            ++it;
        }
        dp_aisle(v, g, a - pa, lo, hi, gap);
        pa = a;
    }
    return !has_o && nt == 0 ? 0 : dp_final(v);
}

__device__ __forceinline__ unsigned long long block_min_u64(unsigned long long x, unsigned long long* red) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) x = min(x, __shfl_xor_sync(0xffffffffu, x, d));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();   // red is free
    if (lane == 0) red[warp] = x;
    __syncthreads();
    unsigned long long r = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = min(r, red[w]);
    return r;
}

__global__ void __launch_bounds__(BG_THREADS) k_batch_grow(BatchGrowArgs B) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long red[BG_THREADS / 32];
    __shared__ int s_na, s_nrem;
    const EvalArgs& a = B.a;
    const Geo& g = a.g;
    const int tid = threadIdx.x, T = blockDim.x;
    const int n_orders = a.n_orders, n_lines = a.n_lines, A = g.A;
    const int p = blockIdx.x;
    // carve shared memory (sizes match batch_grow_smem_bytes)
    unsigned char* q = smem;
    BgShared S;
    S.off = reinterpret_cast<int32_t*>(q);
    q += 4 * (size_t)(n_orders + 1);
    S.alone = reinterpret_cast<int32_t*>(q);
    q += 4 * (size_t)n_orders;
    S.mask = reinterpret_cast<uint32_t*>(q);
    q += 32 * (size_t)A;
    S.rec = reinterpret_cast<uint32_t*>(q);
    q += 4 * (size_t)A;
    S.key = reinterpret_cast<uint16_t*>(q);
    q += 2 * (size_t)n_lines;
    S.alist = reinterpret_cast<uint16_t*>(q);
    q += 2 * (size_t)A;
    S.rem = reinterpret_cast<uint16_t*>(q);
    q += 2 * (size_t)n_orders;
    S.pos = reinterpret_cast<uint16_t*>(q);
    q += 2 * (size_t)n_orders;
    S.n_aisles = &s_na;

    const int32_t* map = a.slot_map + (int64_t)p * a.slot_stride;
    int32_t* tour_off = B.tour_off + (int64_t)p * (n_orders + 1);
    int32_t* order_seq = B.order_seq + (int64_t)p * n_orders;
    bool bad = false;
    for (int o = tid; o <= n_orders; o += T) S.off[o] = a.order_off[o];
    for (int l = tid; l < n_lines; l += T) {
        const int s = a.line_sku[l];
        const int loc = (unsigned)s < (unsigned)a.n_sku ? map[s] : -1;
        if ((unsigned)loc >= (unsigned)g.n_loc) {
            bad = true;
            S.key[l] = 0;
        } else {
            S.key[l] = (uint16_t)key16_of(loc_key(g, loc));
        }
    }
    for (int i = tid; i < 8 * A; i += T) S.mask[i] = 0u;
    for (int o = tid; o < n_orders; o += T) {
        S.rem[o] = (uint16_t)o;
        S.pos[o] = (uint16_t)o;
    }
    if (tid == 0) {
        s_na = 0;
        s_nrem = n_orders;
    }
    if (__syncthreads_or(bad)) {
        if (tid == 0) {
            flag(a.status, WH_STATUS_BAD_LOC);
            B.n_tours[p] = -1;
        }
        return;
    }
    // each order's keys ascending (aisle, slot), once
    for (int o = tid; o < n_orders; o += T) {
        const int lb = S.off[o], le = S.off[o + 1];
        for (int i = lb + 1; i < le; ++i) {
            const uint16_t k = S.key[i];
            int j = i;
            while (j > lb && S.key[j - 1] > k) {
                S.key[j] = S.key[j - 1];
                --j;
            }
            S.key[j] = k;
        }
    }
    __syncthreads();
    // every order's tour alone (the tour is empty)
    for (int o = tid; o < n_orders; o += T) S.alone[o] = cost_with(S, g, o);
    __syncthreads();

    int done = 0, tours = 0;
    if (tid == 0) tour_off[0] = 0;
    while (done < n_orders) {
        // seed: the longest order alone (max alone, then lowest id)
        unsigned long long best = ~0ull;
        const int nr = s_nrem;
        for (int i = tid; i < nr; i += T) {
            const int o = S.rem[i];
            best = min(best, ((unsigned long long)(0x7fffffff - S.alone[o]) << 32) | (uint32_t)o);
        }
        best = block_min_u64(best, red);
        int o_add = (int)(best & 0xFFFFFFFFull);
        int cost = S.alone[o_add];
        int count = 0, lines = 0;
        for (;;) {
            // add o_add to the tour (thread 0), emit it
            __syncthreads();
            if (tid == 0) {
                order_seq[done] = o_add;
                // out of the unassigned list: the last entry takes its place
                const int at = S.pos[o_add], last = S.rem[--s_nrem];
                S.rem[at] = (uint16_t)last;
                S.pos[last] = (uint16_t)at;
                for (int l = S.off[o_add]; l < S.off[o_add + 1]; ++l) {
                    const int ai = S.key[l] >> 8, k = S.key[l] & 0xFF;
                    uint32_t* m = S.mask + ai * 8;
                    bool present = false;
                    for (int w = 0; w < 8; ++w) present |= m[w] != 0u;
                    if (!present) {
                        // insert the aisle into the sorted list
                        int j = s_na++;
                        while (j > 0 && S.alist[j - 1] > ai) {
                            S.alist[j] = S.alist[j - 1];
                            --j;
                        }
                        S.alist[j] = (uint16_t)ai;
                    }
                    m[k >> 5] |= 1u << (k & 31);
                }
                for (int l = S.off[o_add]; l < S.off[o_add + 1]; ++l) {
                    const int ai = S.key[l] >> 8;
                    uint32_t m[8];
                    for (int w = 0; w < 8; ++w) m[w] = S.mask[ai * 8 + w];
                    int lo, hi, gap;
                    mask_stats(m, lo, hi, gap);
                    S.rec[ai] = ((uint32_t)lo << 16) | ((uint32_t)hi << 8) | (uint32_t)gap;
                }
            }
            ++done;
            ++count;
            lines += S.off[o_add + 1] - S.off[o_add];
            __syncthreads();
            if (B.max_orders > 0 && count >= B.max_orders) break;
            // grow: the fitting order that lengthens the tour least (the
            // minimum of (increase, id) does not depend on the list's order)
            best = ~0ull;
            const int nrg = s_nrem;
            for (int i = tid; i < nrg; i += T) {
                const int o = S.rem[i];
                if (B.max_lines > 0 && lines + (S.off[o + 1] - S.off[o]) > B.max_lines) continue;
                const int c = cost_with(S, g, o);
                best = min(best, ((unsigned long long)(uint32_t)(c - cost) << 32) | (uint32_t)o);
            }
            best = block_min_u64(best, red);
            if (best == ~0ull) break;
            o_add = (int)(best & 0xFFFFFFFFull);
            cost += (int)(best >> 32);
        }
        // close the tour: clear its masks
        ++tours;
        if (tid == 0) tour_off[tours] = done;
        const int na = s_na;
        for (int i = tid; i < na * 8; i += T) S.mask[(int)S.alist[i >> 3] * 8 + (i & 7)] = 0u;
        __syncthreads();
        if (tid == 0) s_na = 0;
        __syncthreads();
    }
    if (tid == 0) B.n_tours[p] = tours;
}

}  // namespace

size_t batch_grow_smem_bytes(int n_orders, int n_lines, int A) {
    return 4 * (size_t)(n_orders + 1) + 4 * (size_t)n_orders + 32 * (size_t)A + 4 * (size_t)A + 2 * (size_t)n_lines +
           2 * (size_t)A + 4 * (size_t)n_orders + 16;
}

cudaError_t launch_batch_grow(const BatchGrowArgs& B, int n_maps, cudaStream_t s) {
    if (n_maps <= 0) return cudaSuccess;
    const size_t smem = batch_grow_smem_bytes(B.a.n_orders, B.a.n_lines, B.a.g.A);
    cudaError_t e = cudaFuncSetAttribute(k_batch_grow, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_batch_grow<<<n_maps, BG_THREADS, smem, s>>>(B);
    return cudaGetLastError();
}

}  // namespace wh
