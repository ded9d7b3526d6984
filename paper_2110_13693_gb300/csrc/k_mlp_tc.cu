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
#include "tc_common.cuh"

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
// x_full, x_empty, w_full[], w_empty[], acc1, acc2, done, red[2], h1c[4]
constexpr int N_BARS = 2 + 2 * TC_STAGES + 5 + 4;
constexpr uint32_t OFF_MISC = OFF_BAR + 8 * N_BARS;  // TMEM base address, abort flag
constexpr uint32_t TC_SMEM = OFF_MISC + 16 + 1024;   // + slack to align the base to 1024 bytes

// Training forward: the pre-activations (fp32) and activations (bf16) of
// both hidden layers, row-major [n][256], for the backward pass; all NULL for
// inference.
struct MlpSave {
    float* Z1;
    __nv_bfloat16* H1;
    float* Z2;
    __nv_bfloat16* H2;
};

// Test hook of the bounded waits: the producer stops before the tile
// `skip_tile` (so that the MMA warp's wait for its features never completes)
// and every wait gives up after wait_ns.  skip_tile < 0 in normal use.
struct TcFault {
    int64_t skip_tile;
    unsigned long long wait_ns;
};

template <bool SAVE>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_mlp_tc(const __grid_constant__ CUtensorMap mx, const __grid_constant__ CUtensorMap mw1,
             const __grid_constant__ CUtensorMap mw2, const float* __restrict__ P, int64_t n, float* __restrict__ y,
             int* status, MlpSave save, TcFault fault) {
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
    const uint32_t acc1_full = bar0 + 16 + 16 * TC_STAGES, acc2_full = acc1_full + 8, done = acc1_full + 16,
                   red_full = acc1_full + 24;   // red_full: two barriers
    // h1c(c): the layer-1 activations of K-chunk c (columns 64c .. 64c+63)
    // are in shared memory, so layer 2's MMAs on that chunk can start
    auto h1c = [&](int c) { return acc1_full + 40 + 8u * c; };
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
        for (int c = 0; c < 4; ++c) mbar_init(h1c(c), TC_EPI_WARPS * 32);
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
                if (tile == fault.skip_tile) break;   // test hook: nothing of this tile is issued
                if (xs > 0 && !(ok = mbar_wait(x_empty, (xs - 1) & 1u, abort, status, fault.wait_ns))) break;
                mbar_expect_tx(x_full, X_BYTES);
                for (int q = 0; q < 3; ++q) tma_load_2d(sX + q * ATOM, &mx, x_full, 64 * q, (int)(tile * TC_ROWS));
                ++xs;
                for (int c = 0; c < 7; ++c) {
                    const int s = (int)(g % TC_STAGES);
                    const uint32_t use = g / TC_STAGES;
                    if (use > 0 && !(ok = mbar_wait(w_empty(s), (use - 1) & 1u, abort, status, fault.wait_ns))) break;
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
                if (!(ok = mbar_wait(x_full, ph, abort, status, fault.wait_ns))) break;
                // layer 1: acc1 = X W1 (K = 192 in three chunks of 64)
                for (int c = 0; ok && c < 3; ++c, ++g) {
                    const int s = (int)(g % TC_STAGES);
                    if (!(ok = mbar_wait(w_full(s), (g / TC_STAGES) & 1u, abort, status, fault.wait_ns))) break;
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
                // layer 2: acc2 = H1 W2 (K = 256 in four chunks of 64), each
                // chunk as soon as the epilogue has written its columns of H1
                for (int c = 0; ok && c < 4; ++c, ++g) {
                    if (!(ok = mbar_wait(h1c(c), ph, abort, status, fault.wait_ns))) break;
                    tc_fence_after();
                    const int s = (int)(g % TC_STAGES);
                    if (!(ok = mbar_wait(w_full(s), (g / TC_STAGES) & 1u, abort, status, fault.wait_ns))) break;
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
            if (!__all_sync(0xffffffffu, mbar_wait(acc1_full, ph, abort, status, fault.wait_ns))) break;
            tc_fence_after();
            // layer 1 in K-chunk order: every warp takes its 16 columns of
            // chunk kc (64 kc + 16 part_id ..), then hands the chunk over; the
            // TMEM load of the next chunk is in flight while this one is
            // computed
            auto e1_chunk = [&](int kc, const uint32_t (&v)[16]) {
                const int c0 = 64 * kc + 16 * part_id;
#pragma unroll
                for (int g8 = 0; g8 < 2; ++g8) {
                    const int c = c0 + 8 * g8;
                    const ulonglong2 bA = *reinterpret_cast<const ulonglong2*>(par + c);
                    const ulonglong2 bB = *reinterpret_cast<const ulonglong2*>(par + c + 4);
                    const uint64_t bias[4] = {bA.x, bA.y, bB.x, bB.y};
                    uint32_t w[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const uint64_t z = add2(pk(__uint_as_float(v[8 * g8 + 2 * j]),
                                                   __uint_as_float(v[8 * g8 + 2 * j + 1])), bias[j]);
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
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                tc_fence_before();
                mbar_arrive(h1c(kc));
            };
            uint32_t ta[16], tb[16];
            tc_ld16_issue(tmem + lane_addr + (uint32_t)(16 * part_id), ta);
            tc_wait_ld16(ta);
#pragma unroll
            for (int kc = 0; kc < 4; ++kc) {
                uint32_t(&cur)[16] = (kc & 1) ? tb : ta;
                uint32_t(&nxt)[16] = (kc & 1) ? ta : tb;
                if (kc < 3) tc_ld16_issue(tmem + lane_addr + (uint32_t)(64 * (kc + 1) + 16 * part_id), nxt);
                e1_chunk(kc, cur);
                if (kc < 3) tc_wait_ld16(nxt);
            }
            if (!__all_sync(0xffffffffu, mbar_wait(acc2_full, ph, abort, status, fault.wait_ns))) break;
            tc_fence_after();
            // layer 2: this warp's TC_PART_COLS columns in steps of 16, the
            // next step's TMEM load in flight while one is computed
            uint64_t part2 = dup2(0.0f);
            auto e2_step = [&](int c0, const uint32_t (&v)[16]) {
#pragma unroll
                for (int j4 = 0; j4 < 16; j4 += 4) {
                    const ulonglong2 b = *reinterpret_cast<const ulonglong2*>(par + 256 + c0 + j4);
                    const ulonglong2 w3 = *reinterpret_cast<const ulonglong2*>(par + 512 + c0 + j4);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int j = j4 + 2 * h;
                        const uint64_t z = add2(pk(__uint_as_float(v[j]), __uint_as_float(v[j + 1])), h ? b.y : b.x);
                        float g0, g1;
                        upk(gelu2(z), g0, g1);
                        // the layer-2 activations are bf16 values
                        const uint32_t hb = pack_bf16(g0, g1);
                        if (save_rows) {
                            *reinterpret_cast<uint64_t*>(save.Z2 + row * 256 + c0 + j) = z;
                            *reinterpret_cast<uint32_t*>(save.H2 + row * 256 + c0 + j) = hb;
                        }
                        const uint64_t hv = pk(__uint_as_float(hb << 16), __uint_as_float(hb & 0xFFFF0000u));
                        part2 = fma2(hv, h ? w3.y : w3.x, part2);
                    }
                }
            };
            const uint32_t c2 = (uint32_t)(TC_PART_COLS * part_id);
            tc_ld16_issue(tmem + lane_addr + 256u + c2, ta);
            tc_wait_ld16(ta);
#pragma unroll
            for (int st = 0; st < TC_PART_COLS / 16; ++st) {
                uint32_t(&cur)[16] = (st & 1) ? tb : ta;
                uint32_t(&nxt)[16] = (st & 1) ? ta : tb;
                if (st + 1 < TC_PART_COLS / 16) tc_ld16_issue(tmem + lane_addr + 256u + c2 + 16u * (st + 1), nxt);
                e2_step((int)c2 + 16 * st, cur);
                if (st + 1 < TC_PART_COLS / 16) tc_wait_ld16(nxt);
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
                if (!__all_sync(0xffffffffu, mbar_wait(rbar, (uint32_t)(it >> 1) & 1u, abort, status, fault.wait_ns))) break;
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
                          float* Z2, void* H2, int64_t skip_tile, unsigned long long wait_ns) {
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
    TcFault fault;
    fault.skip_tile = skip_tile;
    fault.wait_ns = wait_ns ? wait_ns : WAIT_NS;
    kern<<<grid, TC_THREADS, TC_SMEM, s>>>(mx, mw1, mw2, P, n, y, status, save, fault);
    return cudaGetLastError();
}

}  // namespace wh
