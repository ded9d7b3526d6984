// K-means slotting on the GPU (subproblem 3 of Sec. 5: products placed by
// picking frequency, an unsupervised K-means classification deciding which
// are stored together; subroutine 4 then scores the placement with the
// evaluator).  All arithmetic is integer, so the result is exact:
//   features  co_s = sum over every line of s of (T_o - r_s), T_o the sum of
//             the sign rows of the order's lines (= the co-occurrence row of
//             s projected on the sign directions); x_s = trunc(co_s * 1024 /
//             isqrt(|co_s|^2)), last coordinate freq_weight * bitlen(freq_s);
//   seeding   the given SKUs, or K-means++ (Arthur & Vassilvitskii 2007) from
//             the caller's draws: next seed = first SKU whose running sum of
//             D^2 exceeds u mod sum D^2;
//   Lloyd     nearest centroid (ties: lowest), centroid = member mean rounded
//             to the nearest integer (halves up), empty clusters kept;
//   zones     clusters by picks (heavier first), SKUs by picks inside, the
//             r-th SKU at the r-th location in aisle-major order.
// Distances fit int32: |x_j| <= 1024 for the 31 sketch coordinates and
// 0 <= x_31 <= 32 * 256, so a squared distance is below 31 * 2048^2 + 8192^2
// < 2^31; centroids are means of rows and obey the same bounds.
#include "tour_core.cuh"

namespace wh {

namespace {

constexpr int KM_T = 256;

__device__ __forceinline__ void load_row(const int32_t* p, int32_t (&v)[KM_DIM]) {
    const int4* q = reinterpret_cast<const int4*>(p);
#pragma unroll
    for (int i = 0; i < KM_DIM / 4; ++i) {
        const int4 w = q[i];
        v[4 * i] = w.x;
        v[4 * i + 1] = w.y;
        v[4 * i + 2] = w.z;
        v[4 * i + 3] = w.w;
    }
}

__device__ __forceinline__ void load_signs(const int8_t* p, int32_t (&r)[KM_DIM]) {
    const int4* q = reinterpret_cast<const int4*>(p);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int4 w = q[i];
        const int32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) r[16 * i + 4 * b + c] = (int32_t)(int8_t)((uint32_t)ws[b] >> (8 * c));
    }
}

__device__ __forceinline__ int32_t sqdist32(const int32_t (&x)[KM_DIM], const int32_t* c) {
    int32_t d = 0;
#pragma unroll
    for (int j = 0; j < KM_DIM; ++j) {
        const int32_t e = x[j] - c[j];
        d += e * e;
    }
    return d;
}

__device__ __forceinline__ long long floor_div(long long a, long long b) {   // b > 0
    long long q = a / b;
    if ((a % b) != 0 && a < 0) --q;
    return q;
}

// features, step 1: co-occurrence sketch and pick counts (integer atomics,
// so the sums do not depend on the order of the updates)
__global__ void k_km_cooc(KmArgs A) {
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < A.n_orders; o += gridDim.x * blockDim.x) {
        const int lb = A.order_off[o], le = A.order_off[o + 1];
        if (lb < 0 || le < lb || le > A.n_lines) {
            flag(A.status, WH_STATUS_BAD_OFFSET);
            continue;
        }
        int32_t T[KM_DIM];
#pragma unroll
        for (int j = 0; j < KM_DIM; ++j) T[j] = 0;
        bool bad = false;
        for (int l = lb; l < le; ++l) {
            const int s = A.line_sku[l];
            if ((unsigned)s >= (unsigned)A.n_sku) {
                bad = true;
                continue;
            }
            int32_t r[KM_DIM];
            load_signs(A.signs + (int64_t)s * KM_DIM, r);
#pragma unroll
            for (int j = 0; j < KM_SKETCH; ++j) T[j] += r[j];
        }
        if (bad) flag(A.status, WH_STATUS_BAD_SKU);
        for (int l = lb; l < le; ++l) {
            const int s = A.line_sku[l];
            if ((unsigned)s >= (unsigned)A.n_sku) continue;
            int32_t r[KM_DIM];
            load_signs(A.signs + (int64_t)s * KM_DIM, r);
            atomicAdd(&A.freq[s], 1);
            unsigned long long* co = reinterpret_cast<unsigned long long*>(A.co + (int64_t)s * KM_DIM);
#pragma unroll
            for (int j = 0; j < KM_SKETCH; ++j) {
                const int32_t v = T[j] - r[j];
                if (v != 0) atomicAdd(co + j, (unsigned long long)(long long)v);
            }
        }
    }
}

__device__ __forceinline__ long long isqrt_ll(long long v) {
    long long r = (long long)sqrt((double)v);
    while (r > 0 && r * r > v) --r;
    while ((r + 1) * (r + 1) <= v) ++r;
    return r;
}

// features, step 2: normalise the sketch, append the frequency coordinate
__global__ void k_km_features(KmArgs A) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= A.n_sku) return;
    const long long* co = A.co + (int64_t)s * KM_DIM;
    long long c[KM_SKETCH];
    long long nn = 0;
#pragma unroll
    for (int j = 0; j < KM_SKETCH; ++j) {
        c[j] = co[j];
        nn += c[j] * c[j];
    }
    const long long n = isqrt_ll(nn);
    int32_t x[KM_DIM];
#pragma unroll
    for (int j = 0; j < KM_SKETCH; ++j) x[j] = n > 0 ? (int32_t)(c[j] * KM_SCALE / n) : 0;
    const int f = A.freq[s];
    x[KM_SKETCH] = A.fw * (f > 0 ? 32 - __clz(f) : 0);
    int4* out = reinterpret_cast<int4*>(A.x + (int64_t)s * KM_DIM);
#pragma unroll
    for (int i = 0; i < KM_DIM / 4; ++i) out[i] = make_int4(x[4 * i], x[4 * i + 1], x[4 * i + 2], x[4 * i + 3]);
}

// seeds given: copy them (range-checked)
__global__ void k_km_seed_copy(KmArgs A) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= A.k) return;
    int s = A.init[c];
    if ((unsigned)s >= (unsigned)A.n_sku) {
        flag(A.status, WH_STATUS_BAD_SKU);
        s = 0;
    }
    A.seeds[c] = s;
}

__global__ void k_km_pp_first(KmArgs A) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        A.seeds[0] = (int32_t)(A.u[0] % (unsigned long long)A.n_sku);
        *A.done = 0u;
    }
}

__device__ __forceinline__ long long block_sum_ll(long long v, long long* red) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    long long t = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    return t;
}

// inclusive block scan of int64 values
__device__ __forceinline__ long long block_scan_ll(long long v, long long* red) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    long long x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    __syncthreads();
    if (lane == 31) red[w] = x;
    __syncthreads();
    long long before = 0;
    for (int i = 0; i < w; ++i) before += red[i];
    return before + x;
}

// K-means++ round c >= 1: fold seed c-1 into D, then the last block to finish
// draws seed c from the running sums of D (in SKU order)
__global__ void __launch_bounds__(KM_T) k_km_pp_round(KmArgs A, int c) {
    __shared__ long long red[KM_T / 32];
    __shared__ bool last;
    __shared__ long long s_target, s_before;
    __shared__ int s_block, s_pick;
    const int s = blockIdx.x * KM_T + threadIdx.x;
    const int ctr = A.seeds[c - 1];
    long long dm = 0;
    if (s < A.n_sku) {
        int32_t x[KM_DIM], y[KM_DIM];
        load_row(A.x + (int64_t)s * KM_DIM, x);
        load_row(A.x + (int64_t)ctr * KM_DIM, y);
        const long long d = sqdist32(x, y);
        dm = min(A.dmin[s], d);
        A.dmin[s] = dm;
    }
    const long long bs = block_sum_ll(dm, red);
    if (threadIdx.x == 0) {
        A.bsum[blockIdx.x] = bs;
        __threadfence();
        const unsigned t = atomicAdd(A.done, 1u);
        last = t == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // the block holding the draw: every thread sums a contiguous run of the
    // block sums, a block scan of the runs gives each run's start, and the
    // thread whose run covers the target finds the block inside it
    const int nb = (int)gridDim.x, per = (nb + KM_T - 1) / KM_T;
    const int b0 = min((int)threadIdx.x * per, nb), b1 = min(b0 + per, nb);
    long long part = 0;
    for (int b = b0; b < b1; ++b) part += __ldcg(A.bsum + b);
    const long long incl = block_scan_ll(part, red);
    __shared__ long long s_total;
    if (threadIdx.x == KM_T - 1) s_total = incl;
    if (threadIdx.x == 0) s_pick = -1;
    __syncthreads();
    const long long tot = s_total;
    if (tot == 0) {
        if (threadIdx.x == 0) s_pick = (int)(A.u[c] % (unsigned long long)A.n_sku);
    } else {
        const long long target = (long long)(A.u[c] % (unsigned long long)tot);
        const long long excl = incl - part;
        if (part > 0 && excl <= target && target < incl) {
            long long run = excl;
            int b = b0;
            for (; b < b1; ++b) {
                const long long v = __ldcg(A.bsum + b);
                if (run + v > target) break;
                run += v;
            }
            s_block = b;
            s_before = run;
            s_target = target;
        }
    }
    __syncthreads();
    if (s_pick < 0) {
        const int q = s_block * KM_T + threadIdx.x;
        const long long v = q < A.n_sku ? __ldcg(A.dmin + q) : 0;
        const long long incl = s_before + block_scan_ll(v, red);
        // the first SKU whose running sum exceeds the target
        const bool hit = q < A.n_sku && incl > s_target && incl - v <= s_target;
        if (hit) s_pick = q;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        A.seeds[c] = s_pick >= 0 ? s_pick : A.n_sku - 1;
        *A.done = 0u;
    }
}

__global__ void k_km_gather(KmArgs A) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.k * KM_DIM) return;
    const int c = i / KM_DIM, j = i % KM_DIM;
    A.cent[i] = A.x[(int64_t)A.seeds[c] * KM_DIM + j];
}

// |c|^2 - 2 x.c: the squared distance less |x|^2, a constant per row, so the
// nearest centroid and its ties are the same; fits int32 by the same bounds
__device__ __forceinline__ int32_t dist_less_norm(const int32_t (&x)[KM_DIM], const int32_t* c, int32_t cn) {
    int32_t dot = 0;
#pragma unroll
    for (int j = 0; j < KM_DIM; ++j) dot += x[j] * c[j];
    return cn - 2 * dot;
}

// assignment: nearest centroid per SKU; mode 0 accumulates the member sums
// and counts for the update, mode 1 writes the final assignment, the counts
// and the clusters' pick weights.  Per-block partial sums in shared memory.
__global__ void __launch_bounds__(KM_T) k_km_assign(KmArgs A, int mode) {
    extern __shared__ __align__(16) int32_t sm[];
    const int K = A.k;
    int32_t* cent = sm;                                       // [K][32]
    int32_t* psum = cent + K * KM_DIM;                        // [K][32] (mode 0)
    int32_t* pcnt = psum + K * KM_DIM;                        // [K]
    int32_t* cnorm = pcnt + K;                                // [K] |c|^2
    unsigned long long* pw = reinterpret_cast<unsigned long long*>(cnorm + K);   // [K] (mode 1); 66K ints before it, 8-byte aligned
    for (int i = threadIdx.x; i < K * KM_DIM; i += KM_T) {
        cent[i] = A.cent[i];
        psum[i] = 0;
    }
    for (int i = threadIdx.x; i < K; i += KM_T) {
        pcnt[i] = 0;
        pw[i] = 0ull;
        int32_t nn = 0;
        for (int j = 0; j < KM_DIM; ++j) {
            const int32_t v = A.cent[i * KM_DIM + j];
            nn += v * v;
        }
        cnorm[i] = nn;
    }
    __syncthreads();
    const int s = blockIdx.x * KM_T + threadIdx.x;
    if (s < A.n_sku) {
        int32_t x[KM_DIM];
        load_row(A.x + (int64_t)s * KM_DIM, x);
        int best = 0;
        int32_t bd = dist_less_norm(x, cent, cnorm[0]);
        for (int c = 1; c < K; ++c) {
            const int32_t d = dist_less_norm(x, cent + c * KM_DIM, cnorm[c]);
            if (d < bd) {
                bd = d;
                best = c;
            }
        }
        atomicAdd(&pcnt[best], 1);
        if (mode == 0) {
#pragma unroll
            for (int j = 0; j < KM_DIM; ++j)
                if (x[j] != 0) atomicAdd(&psum[best * KM_DIM + j], x[j]);
        } else {
            A.assign[s] = best;
            atomicAdd(&pw[best], (unsigned long long)A.freq[s]);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < K; i += KM_T) {
        if (pcnt[i]) atomicAdd(&A.cnt[i], pcnt[i]);
        if (mode == 1 && pw[i]) atomicAdd(reinterpret_cast<unsigned long long*>(A.weight) + i, pw[i]);
    }
    if (mode == 0)
        for (int i = threadIdx.x; i < K * KM_DIM; i += KM_T)
            if (psum[i]) atomicAdd(reinterpret_cast<unsigned long long*>(A.sum) + i, (unsigned long long)(long long)psum[i]);
}

__global__ void k_km_update(KmArgs A) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.k * KM_DIM) return;
    const long long n = A.cnt[i / KM_DIM];
    if (n > 0) A.cent[i] = (int32_t)floor_div(2 * A.sum[i] + n, 2 * n);
}

// zones: cluster ranks (heavier first, ties lowest id) and each cluster's
// first position in the SKU order
__global__ void k_km_order(KmArgs A) {
    __shared__ long long w[KM_MAX_K];
    __shared__ int cnt[KM_MAX_K], rank[KM_MAX_K];
    const int K = A.k, c = threadIdx.x;
    if (c < K) {
        w[c] = A.weight[c];
        cnt[c] = A.cnt[c];
    }
    __syncthreads();
    if (c < K) {
        int r = 0;
        for (int d = 0; d < K; ++d) r += (w[d] > w[c]) || (w[d] == w[c] && d < c);
        rank[c] = r;
    }
    __syncthreads();
    if (c < K) {
        int off = 0;
        for (int d = 0; d < K; ++d) off += rank[d] < rank[c] ? cnt[d] : 0;
        A.off[c] = off;
        A.cur[c] = 0;
        A.off_by_rank[rank[c]] = off;
    }
    if (c == 0) A.off_by_rank[K] = A.n_sku;
}

// members of every cluster, contiguous in cluster-rank order (any order
// inside a cluster); key = (picks descending, id ascending)
__global__ void k_km_bucket(KmArgs A) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= A.n_sku) return;
    const int c = A.assign[s];
    const int pos = A.off[c] + atomicAdd(&A.cur[c], 1);
    A.mkey[pos] = ((unsigned long long)(0xFFFFFFFFu - (uint32_t)A.freq[s]) << 32) | (uint32_t)s;
}

// the SKU at position p takes rank lo + (members of its cluster with a
// smaller key); the cluster's keys stream through shared memory in tiles
__global__ void __launch_bounds__(KM_T) k_km_place(KmArgs A) {
    __shared__ unsigned long long tile[KM_T];
    const int p = blockIdx.x * KM_T + threadIdx.x;
    const int n = A.n_sku;
    const bool act = p < n;
    unsigned long long my = 0;
    int lo = 0, hi = 0;
    if (act) {
        my = A.mkey[p];
        int a = 0, b = A.k - 1;   // last rank r with off_by_rank[r] <= p
        while (a < b) {
            const int m = (a + b + 1) >> 1;
            if (A.off_by_rank[m] <= p) a = m; else b = m - 1;
        }
        lo = A.off_by_rank[a];
        hi = A.off_by_rank[a + 1];
    }
    // the union of the block's cluster ranges
    __shared__ int s_lo, s_hi;
    if (threadIdx.x == 0) {
        s_lo = 0x7fffffff;
        s_hi = 0;
    }
    __syncthreads();
    if (act) {
        atomicMin(&s_lo, lo);
        atomicMax(&s_hi, hi);
    }
    __syncthreads();
    const int u0 = s_lo, u1 = s_hi;
    int cntless = 0;
    for (int base = u0; base < u1; base += KM_T) {
        const int q = base + threadIdx.x;
        tile[threadIdx.x] = q < u1 ? A.mkey[q] : ~0ull;
        __syncthreads();
        const int t0 = max(lo - base, 0), t1 = min(hi - base, KM_T);
        for (int t = t0; t < t1; ++t) cntless += tile[t] < my;
        __syncthreads();
    }
    if (!act) return;
    const int r = lo + cntless;
    const int L = A.g.L;
    const int aisle = r / (2 * L), q = r % (2 * L);
    A.slot_map[(uint32_t)my] = (aisle * 2 + (q & 1)) * L + (q >> 1);
}

}  // namespace

size_t kmeans_assign_smem(int k) { return (size_t)(2 * k * KM_DIM + 2 * k) * 4 + (size_t)k * 8 + 16; }

cudaError_t launch_kmeans(const KmArgs& A, cudaStream_t s) {
    const int n = A.n_sku, K = A.k;
    const int gb = (n + KM_T - 1) / KM_T;
    cudaError_t e;
    // features
    if ((e = cudaMemsetAsync(A.co, 0, sizeof(long long) * (size_t)n * KM_DIM, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(A.freq, 0, sizeof(int32_t) * (size_t)n, s)) != cudaSuccess) return e;
    if (A.n_orders > 0) k_km_cooc<<<(A.n_orders + KM_T - 1) / KM_T, KM_T, 0, s>>>(A);
    k_km_features<<<gb, KM_T, 0, s>>>(A);
    // seeds
    if (A.init) {
        k_km_seed_copy<<<(K + KM_T - 1) / KM_T, KM_T, 0, s>>>(A);
    } else {
        k_km_pp_first<<<1, 32, 0, s>>>(A);
        if ((e = cudaMemsetAsync(A.dmin, 0x7F, sizeof(long long) * (size_t)n, s)) != cudaSuccess) return e;
        for (int c = 1; c < K; ++c) k_km_pp_round<<<gb, KM_T, 0, s>>>(A, c);
    }
    k_km_gather<<<(K * KM_DIM + KM_T - 1) / KM_T, KM_T, 0, s>>>(A);
    // Lloyd rounds
    const size_t smem = kmeans_assign_smem(K);
    if ((e = cudaFuncSetAttribute(k_km_assign, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
        return e;
    for (int it = 0; it < A.iters; ++it) {
        if ((e = cudaMemsetAsync(A.sum, 0, sizeof(long long) * (size_t)K * KM_DIM, s)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(A.cnt, 0, sizeof(int32_t) * (size_t)K, s)) != cudaSuccess) return e;
        k_km_assign<<<gb, KM_T, smem, s>>>(A, 0);
        k_km_update<<<(K * KM_DIM + KM_T - 1) / KM_T, KM_T, 0, s>>>(A);
    }
    // final assignment, weights, zones
    if ((e = cudaMemsetAsync(A.cnt, 0, sizeof(int32_t) * (size_t)K, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(A.weight, 0, sizeof(long long) * (size_t)K, s)) != cudaSuccess) return e;
    k_km_assign<<<gb, KM_T, smem, s>>>(A, 1);
    k_km_order<<<1, KM_MAX_K, 0, s>>>(A);
    k_km_bucket<<<gb, KM_T, 0, s>>>(A);
    k_km_place<<<gb, KM_T, 0, s>>>(A);
    return cudaGetLastError();
}

}  // namespace wh
