// Surrogate feature rows, shared by the feature kernels of every tour and of
// the moved tours: a per-warp table of a tour's visited aisles and the
// histograms built from it.  Included by those translation units after
// tour_core.cuh; everything lives in an unnamed namespace.
#pragma once
#include <cuda_bf16.h>

#include "tour_core.cuh"

namespace wh {
namespace {

// ------------------------------------------------------ surrogate features
// 192 features of a tour (the surrogate's input): histograms over its
// visited aisles of the deepest and shallowest pick's slot bin
// floor(k*64/L), leftmost / rightmost aisle and aisle count times 1/A, line
// count / 64, and a 60-bin histogram of the visited aisles floor(a*60/A).
// Bins use exact multiply-shift division: floor(n/d) = (n * ceil(2^40/d)) >> 40
// for n < 2^22 and d < 2^16.
//
// Warp-cooperative: the lanes of a warp gather a tour's lines
// in parallel (one order per lane) and merge the picks into a per-warp
// open-addressing table of visited aisles (shared-memory atomics keep each
// aisle's smallest and largest slot index); the table then feeds the
// histograms and the four scalars, written as one coalesced 384-byte row.
constexpr int WF_SLOTS = 128;    // distinct aisles per tour

struct __align__(16) WarpFeat {
    uint32_t key[WF_SLOTS];     // aisle + 1, 0 = empty
    uint32_t lo[WF_SLOTS];      // smallest slot index seen, 0xFFFFFFFF = none
    uint32_t hi[WF_SLOTS];      // largest slot index seen
    uint32_t cnt[WH_FEATURES];  // histogram counters
};

__device__ __forceinline__ void wf_init(WarpFeat& w, int lane) {
    for (int i = lane; i < WF_SLOTS; i += 32) {
        w.key[i] = 0u;
        w.lo[i] = 0xFFFFFFFFu;
        w.hi[i] = 0u;
    }
    for (int i = lane; i < WH_FEATURES; i += 32) w.cnt[i] = 0u;
    __syncwarp();
}

// Merge one pick (key32 = aisle << 16 | slot index); false when the tour
// visits more than WF_SLOTS aisles.
__device__ __forceinline__ bool wf_insert(WarpFeat& w, uint32_t key32) {
    const uint32_t a = key32 >> 16, k = key32 & 0xFFu;
    uint32_t h = (a * 2654435761u) >> 25;   // 7 bits
    for (int probe = 0; probe < WF_SLOTS; ++probe) {
        const uint32_t old = atomicCAS(&w.key[h], 0u, a + 1u);
        if (old == 0u || old == a + 1u) {
            atomicMin(&w.lo[h], k);
            atomicMax(&w.hi[h], k);
            return true;
        }
        h = (h + 1u) & (WF_SLOTS - 1);
    }
    return false;
}

__device__ __forceinline__ uint32_t feat_div(uint32_t n, uint64_t magic) {
    return (uint32_t)(((uint64_t)n * magic) >> 40);
}

// Write the tour's 192 bf16 features to row (16-byte aligned, lanes 0..23
// write 16 bytes each) and leave the table and counters empty.  n_lines is
// the warp's total line count.  Lane L's eight counters are read and cleared
// as two 16-byte words (eight scalar accesses at a stride of eight words
// would meet six-way bank conflicts).
__device__ __forceinline__ void wf_finish(WarpFeat& w, const FeatConst& c, int lane, uint32_t n_lines, uint4* row) {
    __syncwarp();
    int amin = 0x7fffffff, amax = -1, na = 0;
    for (int i = lane; i < WF_SLOTS; i += 32) {
        const uint32_t kv = w.key[i];
        if (kv == 0u) continue;
        const int a = (int)kv - 1;
        const uint32_t lo = w.lo[i], hi = w.hi[i];
        atomicAdd(&w.cnt[feat_div(hi * 64u, c.magic_l)], 1u);
        atomicAdd(&w.cnt[64 + feat_div(lo * 64u, c.magic_l)], 1u);
        atomicAdd(&w.cnt[132 + feat_div((uint32_t)a * 60u, c.magic_a)], 1u);
        amin = min(amin, a);
        amax = max(amax, a);
        ++na;
        w.key[i] = 0u;
        w.lo[i] = 0xFFFFFFFFu;
        w.hi[i] = 0u;
    }
    amin = __reduce_min_sync(0xffffffffu, amin);
    amax = __reduce_max_sync(0xffffffffu, amax);
    na = (int)__reduce_add_sync(0xffffffffu, (unsigned)na);
    __syncwarp();
    if (lane < 24) {
        uint4* c4 = reinterpret_cast<uint4*>(w.cnt) + 2 * lane;
        const uint4 c0 = c4[0], c1 = c4[1];
        c4[0] = make_uint4(0u, 0u, 0u, 0u);
        c4[1] = make_uint4(0u, 0u, 0u, 0u);
        float v[8] = {(float)c0.x, (float)c0.y, (float)c0.z, (float)c0.w,
                      (float)c1.x, (float)c1.y, (float)c1.z, (float)c1.w};
        if (lane == 16) {   // features 128..131: the four scalars
            v[0] = na ? (float)amin * c.inv_a : 0.0f;
            v[1] = na ? (float)amax * c.inv_a : 0.0f;
            v[2] = (float)na * c.inv_a;
            v[3] = (float)n_lines * (1.0f / 64.0f);
        }
        uint4 o;
        __nv_bfloat162 p0 = __floats2bfloat162_rn(v[0], v[1]), p1 = __floats2bfloat162_rn(v[2], v[3]);
        __nv_bfloat162 p2 = __floats2bfloat162_rn(v[4], v[5]), p3 = __floats2bfloat162_rn(v[6], v[7]);
        o.x = *reinterpret_cast<uint32_t*>(&p0);
        o.y = *reinterpret_cast<uint32_t*>(&p1);
        o.z = *reinterpret_cast<uint32_t*>(&p2);
        o.w = *reinterpret_cast<uint32_t*>(&p3);
        row[lane] = o;
    }
    __syncwarp();
}

}  // namespace
}  // namespace wh
