// Surrogate inference on the 5th-generation tensor cores (tcgen05, sm_103a):
// y = w3 . gelu(W2^T gelu(W1^T x + b1) + b2) + b3 for every row x of the
// bf16 feature matrix, fused in one persistent kernel.  The learned prescreen
// scores every tour and every re-costed tour of a local-search step with this
// network (machine learning in the decision loop, Sec. 1 and Fig. 1).
//
// One CTA per SM; per 128-row tile:
//   producer warp   TMA (cp.async.bulk.tensor, 128-byte swizzle) of the
//                   tile's features [128 x 192] and of the transposed bf16
//                   weights in K-chunks of 64 ([256 x 64] per chunk) through
//                   a 3-stage ring;
//   MMA warp        tcgen05.mma kind::f16 (M 128, N 256, K 16) into two fp32
//                   TMEM accumulators (layer 1 at column 0, layer 2 at 256);
//   16 epilogue warps tcgen05.ld of the accumulators, bias + GELU (erf form,
//                   erf by Abramowitz & Stegun 7.1.28, packed fp32x2 math),
//                   bf16 rounding, the layer-1 activations written back to
//                   shared memory as the next A operand (same swizzle), and
//                   the final dot product with w3.
// Layer 1 of the next tile runs on the tensor cores while the epilogue
// finishes the current one.  The bf16 rounding points equal the training
// path's: activations are rounded to bf16 after each GELU, products
// accumulate in fp32.
//
// Every wait is bounded (about two seconds of %globaltimer): a wait that
// runs out sets the CTA's abort flag and the caller's status word, the other
// roles leave their loops, outstanding copies and MMAs are waited for (again
// bounded), and the TMEM is freed before the CTA exits.
#include <cuda.h>
#include <cuda_bf16.h>

#include "wh_internal.h"

namespace wh {

namespace {

constexpr int TC_ROWS = 128;                      // rows per tile (MMA M)
constexpr int TC_EPI_WARPS = 16;                 // four per TMEM lane quarter
constexpr int TC_PARTS = TC_EPI_WARPS / 4;        // column parts per row
constexpr int TC_PART_COLS = 256 / TC_PARTS;
constexpr int TC_PRODUCER = TC_EPI_WARPS;         // warp index
constexpr int TC_MMA = TC_EPI_WARPS + 1;          // warp index
constexpr int TC_THREADS = (TC_EPI_WARPS + 2) * 32;
constexpr int TC_STAGES = 3;
constexpr uint32_t ATOM = 128 * 128;              // one 128-row K-atom: 128 rows x 64 bf16
constexpr uint32_t X_BYTES = 3 * ATOM;            // [128 x 192]
constexpr uint32_t W_CHUNK = 256 * 128;           // [256 x 64]
constexpr uint32_t H_BYTES = 4 * ATOM;            // [128 x 256]
constexpr uint32_t OFF_X = 0;
constexpr uint32_t OFF_W = OFF_X + X_BYTES;
constexpr uint32_t OFF_H = OFF_W + TC_STAGES * W_CHUNK;
constexpr uint32_t OFF_PAR = OFF_H + H_BYTES;     // b1, b2, w3 (fp32)
constexpr uint32_t OFF_RED = OFF_PAR + 3 * 256 * 4;  // [2 tiles][parts 1..][128] fp32 partial sums
constexpr uint32_t OFF_BAR = OFF_RED + 2 * (TC_PARTS - 1) * 128 * 4;
// x_full, x_empty, w_full[], w_empty[], acc1, h1, acc2, done, red[2]
constexpr int N_BARS = 2 + 2 * TC_STAGES + 6;
constexpr uint32_t OFF_MISC = OFF_BAR + 8 * N_BARS;  // TMEM base address, abort flag
constexpr uint32_t TC_SMEM = OFF_MISC + 16 + 1024;   // + slack to align the base to 1024 bytes

// instruction descriptor of tcgen05.mma kind::f16: fp32 accumulator (bits
// 4-5), A and B bf16 (bits 7-9, 10-12), both K-major (bits 15, 16 clear),
// N/8 at bits 17-22, M/16 at bits 24-28
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((256u >> 3) << 17) | ((128u >> 4) << 24);

constexpr unsigned long long WAIT_NS = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of `parity` to complete.  Gives up when the CTA's abort
// flag is set or after WAIT_NS, setting the flag and the status word.
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort, int* status) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t i = 1;; ++i) {
        if (mbar_try(bar, parity)) return true;
        if ((i & 63) == 0) {
            if (*abort) return false;
            if (globaltimer() - t0 > WAIT_NS || i > (1u << 30)) {
                *abort = 1;
                atomicOr(status, (int)WH_STATUS_TIMEOUT);
                return false;
            }
        }
    }
}

// used after an abort: wait for a phase without giving up on the flag
__device__ void mbar_drain(uint32_t bar, uint32_t parity) {
    const uint64_t t0 = globaltimer();
    for (uint32_t i = 0; !mbar_try(bar, parity); ++i)
        if ((i & 63) == 0 && globaltimer() - t0 > WAIT_NS) return;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], "
        "[%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(IDESC), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// Shared-memory matrix descriptor of a K-major operand in the 128-byte
// swizzled layout that TMA writes: 8-row groups 1024 bytes apart (stride
// byte offset), descriptor version 1 (bit 46), swizzle mode 2 (bits 61-63).
// Advancing K by 16 bf16 inside a 1024-byte aligned atom adds 32 bytes to
// the start address.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// 32 TMEM lanes x 32 fp32 columns: lane i of the warp receives its lane's
// columns [col, col + 32).  The wait names the registers so that no use of
// them is scheduled before the load has landed.
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                   "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                   "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// Pairs of fp32 values in one 64-bit register for the packed fp32x2
// arithmetic of sm_100 and later (add / mul / fma .f32x2, element-wise,
// round to nearest): the epilogue's FMA-pipe work in half the instructions.
__device__ __forceinline__ uint64_t pk(float lo, float hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk(uint64_t r, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(r));
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t dup2(float x) { return pk(x, x); }

// gelu(z) = z/2 (1 + erf(z / sqrt 2)) of both halves of z.  erf by the
// approximation of Abramowitz & Stegun, Handbook of Mathematical Functions,
// formula 7.1.28 (after Hastings): for x >= 0,
// erf(x) = 1 - (1 + a1 x + a2 x^2 + ... + a6 x^6)^-16, |error| <= 3e-7; odd
// in x (large x: the power overflows to inf and erf to 1).  Far below the
// bf16 resolution (2^-8) of the activations it feeds; one reciprocal per
// value and FMAs, all but the reciprocal on packed pairs.
__device__ __forceinline__ uint64_t gelu2(uint64_t z) {
    float x0, x1;
    upk(mul2(z, dup2(0.70710678118654752f)), x0, x1);
    const uint64_t ax = pk(fabsf(x0), fabsf(x1));
    uint64_t p = fma2(dup2(0.0000430638f), ax, dup2(0.0002765672f));
    p = fma2(p, ax, dup2(0.0001520143f));
    p = fma2(p, ax, dup2(0.0092705272f));
    p = fma2(p, ax, dup2(0.0422820123f));
    p = fma2(p, ax, dup2(0.0705230784f));
    p = fma2(p, ax, dup2(1.0f));
    p = mul2(p, p);   // ^2
    p = mul2(p, p);   // ^4
    p = mul2(p, p);   // ^8
    p = mul2(p, p);   // ^16
    float p0, p1;
    upk(p, p0, p1);
    const float m0 = 1.0f - 1.0f / p0, m1 = 1.0f - 1.0f / p1;   // |erf|
    const uint64_t er = pk(copysignf(m0, x0), copysignf(m1, x1));
    const uint64_t hz = mul2(z, dup2(0.5f));
    return fma2(hz, er, hz);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 p = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&p);
}

// Training forward: the pre-activations (fp32) and activations (bf16) of
// both hidden layers, row-major [n][256], for the backward pass; all NULL for
// inference.
struct MlpSave {
    float* Z1;
    __nv_bfloat16* H1;
    float* Z2;
    __nv_bfloat16* H2;
};

template <bool SAVE>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_mlp_tc(const __grid_constant__ CUtensorMap mx, const __grid_constant__ CUtensorMap mw1,
             const __grid_constant__ CUtensorMap mw2, const float* __restrict__ P, int64_t n, float* __restrict__ y,
             int* status, MlpSave save) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t sX = sbase + OFF_X, sW = sbase + OFF_W, sH = sbase + OFF_H;
    float* par = reinterpret_cast<float*>(smem + OFF_PAR);   // b1[256] b2[256] w3[256]
    float* red = reinterpret_cast<float*>(smem + OFF_RED);
    const uint32_t bar0 = sbase + OFF_BAR;
    const uint32_t x_full = bar0, x_empty = bar0 + 8;
    auto w_full = [&](int s) { return bar0 + 16 + 8u * s; };
    auto w_empty = [&](int s) { return bar0 + 16 + 8u * (TC_STAGES + s); };
    const uint32_t acc1_full = bar0 + 16 + 16 * TC_STAGES, h1_full = acc1_full + 8, acc2_full = acc1_full + 16,
                   done = acc1_full + 24, red_full = acc1_full + 32;   // red_full: two barriers
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + OFF_MISC);
    volatile int* abort = reinterpret_cast<volatile int*>(smem + OFF_MISC + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t n_tiles = (n + TC_ROWS - 1) / TC_ROWS;

    for (int i = threadIdx.x; i < 768; i += TC_THREADS)
        par[i] = i < 256 ? P[MLP_B1_OFF + i] : i < 512 ? P[MLP_B2_OFF + i - 256] : P[MLP_W3_OFF + i - 512];
    if (threadIdx.x == 0) {
        *abort = 0;
        mbar_init(x_full, 1);
        mbar_init(x_empty, 1);
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(w_full(s), 1);
            mbar_init(w_empty(s), 1);
        }
        mbar_init(acc1_full, 1);
        mbar_init(h1_full, TC_EPI_WARPS * 32);
        mbar_init(acc2_full, 1);
        mbar_init(done, 1);
        mbar_init(red_full, (TC_PARTS - 1) * 128);
        mbar_init(red_full + 8, (TC_PARTS - 1) * 128);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == TC_MMA) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == TC_PRODUCER) {
        if (lane == 0) {
            uint32_t g = 0, xs = 0;   // weight chunks and feature tiles issued
            bool ok = true;
            for (int64_t tile = blockIdx.x; ok && tile < n_tiles; tile += gridDim.x) {
                if (xs > 0 && !(ok = mbar_wait(x_empty, (xs - 1) & 1u, abort, status))) break;
                mbar_expect_tx(x_full, X_BYTES);
                for (int q = 0; q < 3; ++q) tma_load_2d(sX + q * ATOM, &mx, x_full, 64 * q, (int)(tile * TC_ROWS));
                ++xs;
                for (int c = 0; c < 7; ++c) {
                    const int s = (int)(g % TC_STAGES);
                    const uint32_t use = g / TC_STAGES;
                    if (use > 0 && !(ok = mbar_wait(w_empty(s), (use - 1) & 1u, abort, status))) break;
                    mbar_expect_tx(w_full(s), W_CHUNK);
                    if (c < 3) tma_load_2d(sW + s * W_CHUNK, &mw1, w_full(s), 64 * c, 0);
                    else tma_load_2d(sW + s * W_CHUNK, &mw2, w_full(s), 64 * (c - 3), 0);
                    ++g;
                }
            }
            if (*abort) {
                // let the copies still in flight land before the CTA exits:
                // only the last fill of each barrier can be outstanding
                if (xs > 0) mbar_drain(x_full, (xs - 1) & 1u);
                for (uint32_t k = 0; k < TC_STAGES && k < g; ++k) {
                    const uint32_t last = g - 1 - k;
                    mbar_drain(w_full((int)(last % TC_STAGES)), (last / TC_STAGES) & 1u);
                }
            }
        }
    } else if (warp == TC_MMA) {
        if (lane == 0) {
            uint32_t g = 0;
            int64_t it = 0;
            bool ok = true;
            const uint32_t acc1 = tmem, acc2 = tmem + 256;
            for (int64_t tile = blockIdx.x; ok && tile < n_tiles; tile += gridDim.x, ++it) {
                const uint32_t ph = (uint32_t)it & 1u;
                if (!(ok = mbar_wait(x_full, ph, abort, status))) break;
                // layer 1: acc1 = X W1 (K = 192 in three chunks of 64)
                for (int c = 0; ok && c < 3; ++c, ++g) {
                    const int s = (int)(g % TC_STAGES);
                    if (!(ok = mbar_wait(w_full(s), (g / TC_STAGES) & 1u, abort, status))) break;
                    tc_fence_after();
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        tc_mma(acc1, sw128_desc(sX + c * ATOM + 32 * kk), sw128_desc(sW + s * W_CHUNK + 32 * kk),
                               (c | kk) != 0);
                    tc_commit(w_empty(s));
                }
                if (!ok) break;
                tc_commit(x_empty);
                tc_commit(acc1_full);
                // layer 2: acc2 = H1 W2 (K = 256 in four chunks of 64), once
                // the epilogue has written H1
                if (!(ok = mbar_wait(h1_full, ph, abort, status))) break;
                tc_fence_after();
                for (int c = 0; ok && c < 4; ++c, ++g) {
                    const int s = (int)(g % TC_STAGES);
                    if (!(ok = mbar_wait(w_full(s), (g / TC_STAGES) & 1u, abort, status))) break;
                    tc_fence_after();
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        tc_mma(acc2, sw128_desc(sH + c * ATOM + 32 * kk), sw128_desc(sW + s * W_CHUNK + 32 * kk),
                               (c | kk) != 0);
                    tc_commit(w_empty(s));
                }
                if (!ok) break;
                tc_commit(acc2_full);
            }
            // every MMA issued has completed once `done` fires
            tc_commit(done);
            mbar_drain(done, 0);
        }
    } else {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (its rows) and
        // the column part w / 4 (TC_PART_COLS columns of each layer)
        const int quarter = warp & 3, part_id = warp >> 2;
        const int r = 32 * quarter + lane;
        const uint32_t lane_addr = (uint32_t)(32 * quarter) << 16;
        const float b3 = P[MLP_B3_OFF];
        int64_t it = 0;
        for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++it) {
            const uint32_t ph = (uint32_t)it & 1u;
            const int64_t row = tile * TC_ROWS + r;
            const bool save_rows = SAVE && row < n;
            // the TMEM loads below are warp-collective: leave together
            if (!__all_sync(0xffffffffu, mbar_wait(acc1_full, ph, abort, status))) break;
            tc_fence_after();
#pragma unroll 1
            for (int cc = 0; cc < TC_PART_COLS / 32; ++cc) {
                const int c0 = TC_PART_COLS * part_id + 32 * cc;
                float v[32];
                tc_ld32(tmem + lane_addr + (uint32_t)c0, v);
#pragma unroll
                for (int g8 = 0; g8 < 4; ++g8) {
                    uint32_t w[4];
                    const int c = c0 + 8 * g8;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const uint64_t b = *reinterpret_cast<const uint64_t*>(par + c + 2 * j);
                        const uint64_t z = add2(pk(v[8 * g8 + 2 * j], v[8 * g8 + 2 * j + 1]), b);
                        if (save_rows) *reinterpret_cast<uint64_t*>(save.Z1 + row * 256 + c + 2 * j) = z;
                        float g0, g1;
                        upk(gelu2(z), g0, g1);
                        w[j] = pack_bf16(g0, g1);
                    }
                    const uint4 o = make_uint4(w[0], w[1], w[2], w[3]);
                    if (save_rows) *reinterpret_cast<uint4*>(save.H1 + row * 256 + c) = o;
                    // 128-byte swizzle: 16-byte chunk j of row r sits at chunk j ^ (r % 8)
                    const int chunk = (c & 63) >> 3;
                    unsigned char* dst = smem + OFF_H + (c >> 6) * ATOM + r * 128 + ((chunk ^ (r & 7)) << 4);
                    *reinterpret_cast<uint4*>(dst) = o;
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tc_fence_before();
            mbar_arrive(h1_full);
            if (!__all_sync(0xffffffffu, mbar_wait(acc2_full, ph, abort, status))) break;
            tc_fence_after();
            uint64_t part2 = dup2(0.0f);
#pragma unroll 1
            for (int cc = 0; cc < TC_PART_COLS / 32; ++cc) {
                const int c0 = TC_PART_COLS * part_id + 32 * cc;
                float v[32];
                tc_ld32(tmem + lane_addr + 256u + (uint32_t)c0, v);
#pragma unroll
                for (int j = 0; j < 32; j += 2) {
                    const uint64_t b = *reinterpret_cast<const uint64_t*>(par + 256 + c0 + j);
                    const uint64_t z = add2(pk(v[j], v[j + 1]), b);
                    float g0, g1;
                    upk(gelu2(z), g0, g1);
                    // the layer-2 activations are bf16 values
                    const uint32_t hb = pack_bf16(g0, g1);
                    if (save_rows) {
                        *reinterpret_cast<uint64_t*>(save.Z2 + row * 256 + c0 + j) = z;
                        *reinterpret_cast<uint32_t*>(save.H2 + row * 256 + c0 + j) = hb;
                    }
                    const uint64_t h = pk(__uint_as_float(hb << 16), __uint_as_float(hb & 0xFFFF0000u));
                    part2 = fma2(h, *reinterpret_cast<const uint64_t*>(par + 512 + c0 + j), part2);
                }
            }
            float pa, pb;
            upk(part2, pa, pb);
            const float part = pa + pb;
            // the other column parts hand their partial sums to part 0, which
            // adds them in a fixed order
            float* rb = red + (it & 1) * (TC_PARTS - 1) * 128;
            const uint32_t rbar = red_full + 8u * (uint32_t)(it & 1);
            if (part_id > 0) {
                rb[(part_id - 1) * 128 + r] = part;
                mbar_arrive(rbar);
            } else {
                if (!__all_sync(0xffffffffu, mbar_wait(rbar, (uint32_t)(it >> 1) & 1u, abort, status))) break;
                float sum = part;
#pragma unroll
                for (int k = 0; k < TC_PARTS - 1; ++k) sum += rb[k * 128 + r];
                if (row < n) y[row] = sum + b3;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == TC_MMA) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    }
}

__global__ void k_transpose_bf16(const float* __restrict__ p, int K, int N, __nv_bfloat16* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= K * N) return;
    const int nn = i / K, k = i - nn * K;   // out[nn][k] = p[k][nn]
    out[i] = __float2bfloat16_rn(p[(int64_t)k * N + nn]);
}

}  // namespace

size_t mlp_tc_smem_bytes() { return TC_SMEM; }

cudaError_t launch_transpose_bf16(const float* p, int K, int N, void* out, cudaStream_t s) {
    const int n = K * N;
    k_transpose_bf16<<<(n + 255) / 256, 256, 0, s>>>(p, K, N, static_cast<__nv_bfloat16*>(out));
    return cudaGetLastError();
}

cudaError_t launch_mlp_tc(const CUtensorMap& mx, const CUtensorMap& mw1, const CUtensorMap& mw2, const float* P,
                          int64_t n, float* y, int* status, int num_sms, cudaStream_t s, float* Z1, void* H1,
                          float* Z2, void* H2) {
    if (n <= 0) return cudaSuccess;
    const bool save_acts = Z1 && H1 && Z2 && H2;
    auto kern = save_acts ? k_mlp_tc<true> : k_mlp_tc<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (n + TC_ROWS - 1) / TC_ROWS;
    const int grid = (int)(tiles < num_sms ? tiles : num_sms);
    MlpSave save;
    save.Z1 = Z1;
    save.H1 = static_cast<__nv_bfloat16*>(H1);
    save.Z2 = Z2;
    save.H2 = static_cast<__nv_bfloat16*>(H2);
    kern<<<grid, TC_THREADS, TC_SMEM, s>>>(mx, mw1, mw2, P, n, y, status, save);
    return cudaGetLastError();
}

}  // namespace wh
