// Surrogate training backward on the 5th-generation tensor cores (tcgen05,
// sm_103a): the gradients of 0.5 * mean((y - t)^2) of the prescreen's MLP
// (machine learning in the decision loop, Sec. 1 and Fig. 1; bf16 weights and
// activations with fp32 accumulation).  After the tensor-core training
// forward (k_mlp_tc.cu, which keeps Z1, H1, Z2, H2):
//
//   k_bwd_tail   32 rows per block: dy = (y - t) / n, the loss, dZ2 =
//                bf16(dy * w3 * gelu'(Z2)) row-major and transposed, H1
//                transposed, X transposed with a row of ones appended (so
//                that the weight gradient of layer 1 also yields the bias
//                gradient), and per-block column sums for b2, w3 and b3;
//   k_mlp_dz1    dZ1 = bf16((dZ2 W2^T) * gelu'(Z1)), 128 rows per tile on
//                tcgen05 (M 128, N 256, K 256; W2 resident in shared memory),
//                written row-major and transposed;
//   k_mlp_wgrad  dW2 = H1^T dZ2 and [dW1; db1] = [X 1]^T dZ1 on tcgen05,
//                the batch (the reduction) split into ranges, one CTA per
//                (product, 128-row tile of the output, range), operands
//                K-major from the transposed copies, fp32 partials;
//   k_adam_parts every gradient as the sum of its partials in a fixed order
//                (deterministic), then Adam on the fp32 master weights and
//                the bf16 copies.
//
// The rounding points equal those of the oracle's training trace: dZ2 and
// dZ1 are rounded to bf16 where they become MMA operands; products
// accumulate in fp32.  Every mbarrier wait is bounded (tc_common.cuh).
#include "tc_common.cuh"

namespace wh {

namespace {

constexpr uint32_t BW_ATOM = 128 * 128;     // one 128-row K-atom: 128 rows x 64 bf16 (128-byte swizzle)
constexpr uint32_t BW_WCHUNK = 256 * 128;   // [256 x 64] bf16
constexpr int BT_ROWS = 32;                 // rows per tail block
constexpr int BT_THREADS = 256;
constexpr int BT_PART = 520;                // floats per tail block: b2[256] g3[256] gb3 loss (padded)
constexpr int BW_EPI0 = 2;                  // first epilogue warp (warps 0, 1: producer, MMA)
constexpr int BW_THREADS = (BW_EPI0 + 4) * 32;

__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// ------------------------------------------------------------------ tail
// The tile s_t[col][row] (rows r0 .. r0+31) written to a transposed copy,
// 64 bytes of each column, 16 at a time.
__device__ __forceinline__ void write_transposed(const __nv_bfloat16 (*s_t)[BT_ROWS + 8], int cols,
                                                 __nv_bfloat16* dst, int64_t ldt, int64_t r0, int tid) {
    for (int c = tid; c < cols * 4; c += BT_THREADS) {
        const int j = c >> 2, q = c & 3;
        *reinterpret_cast<uint4*>(dst + (int64_t)j * ldt + r0 + 8 * q) = *reinterpret_cast<const uint4*>(&s_t[j][8 * q]);
    }
}

__global__ void __launch_bounds__(BT_THREADS) k_bwd_tail(BwdArgs b) {
    __shared__ float s_dy[BT_ROWS];
    __shared__ __align__(16) __nv_bfloat16 s_t[256][BT_ROWS + 8];
    const int tid = threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.x * BT_ROWS;
    float* part = b.part_t + (int64_t)blockIdx.x * BT_PART;
    // H1 transposed (the forward's activations; rows past n are zero)
    {
        const int j = tid;
#pragma unroll 8
        for (int rr = 0; rr < BT_ROWS; ++rr) {
            const int64_t r = r0 + rr;
            s_t[j][rr] = r < b.n ? b.H1[r * 256 + j] : __float2bfloat16_rn(0.0f);
        }
    }
    __syncthreads();
    write_transposed(s_t, 256, b.H1T, b.ldt, r0, tid);
    __syncthreads();
    if (tid < 32) {
        const int64_t r = r0 + tid;
        float d = 0.0f, l = 0.0f;
        if (r < b.n) {
            const float e = b.y[r] - b.t[r];
            d = e / (float)b.n;
            l = 0.5f * e * e / (float)b.n;
            b.dy[r] = d;
        }
        s_dy[tid] = d;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            l += __shfl_xor_sync(0xffffffffu, l, o);
            d += __shfl_xor_sync(0xffffffffu, d, o);
        }
        if (tid == 0) {
            part[512] = d;   // sum of dy: the gradient of b3
            part[513] = l;
        }
    }
    __syncthreads();
    {
        // dZ2 = bf16(dy * w3 * gelu'(Z2)), eight rows' loads in flight
        const int j = tid;
        const float w3j = b.P[MLP_W3_OFF + j];
        float sb2 = 0.0f, sg3 = 0.0f;
        for (int r8 = 0; r8 < BT_ROWS; r8 += 8) {
            float z[8], h[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int64_t r = r0 + r8 + u;
                z[u] = r < b.n ? b.Z2[r * 256 + j] : 0.0f;
                h[u] = r < b.n ? __bfloat162float(b.H2[r * 256 + j]) : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int64_t r = r0 + r8 + u;
                __nv_bfloat16 v = __float2bfloat16_rn(0.0f);
                if (r < b.n) {
                    const float dyr = s_dy[r8 + u];
                    v = __float2bfloat16_rn(dyr * w3j * gelu_grad(z[u]));
                    b.dZ2[r * 256 + j] = v;
                    sb2 += __bfloat162float(v);
                    sg3 += h[u] * dyr;
                }
                s_t[j][r8 + u] = v;
            }
        }
        part[j] = sb2;
        part[256 + j] = sg3;
    }
    __syncthreads();
    write_transposed(s_t, 256, b.dZ2T, b.ldt, r0, tid);
    __syncthreads();
    // X transposed, with row 192 = 1 for every row of the batch
    if (tid <= (int)MLP_IN) {
#pragma unroll 8
        for (int rr = 0; rr < BT_ROWS; ++rr) {
            const int64_t r = r0 + rr;
            __nv_bfloat16 v = __float2bfloat16_rn(0.0f);
            if (r < b.n) v = tid < (int)MLP_IN ? b.X[r * MLP_IN + tid] : __float2bfloat16_rn(1.0f);
            s_t[tid][rr] = v;
        }
    }
    __syncthreads();
    write_transposed(s_t, (int)MLP_IN + 1, b.XT, b.ldt, r0, tid);
}

// ------------------------------------------------------------------- dZ1
// smem: A tile [128 x 256] (four atoms), W2 [256 x 256] (four chunks), bars
constexpr uint32_t D1_OFF_A = 0;
constexpr uint32_t D1_OFF_W = D1_OFF_A + 4 * BW_ATOM;
constexpr uint32_t D1_OFF_BAR = D1_OFF_W + 4 * BW_WCHUNK;
constexpr int D1_NBARS = 6;   // w_full, a_full, a_empty, acc_full, acc_empty, done
constexpr uint32_t D1_OFF_MISC = D1_OFF_BAR + 8 * D1_NBARS;
constexpr uint32_t D1_SMEM = D1_OFF_MISC + 16 + 1024;

__global__ void __launch_bounds__(BW_THREADS, 1)
    k_mlp_dz1(const __grid_constant__ CUtensorMap mdz2, const __grid_constant__ CUtensorMap mw2, BwdArgs b) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t sA = sbase + D1_OFF_A, sW = sbase + D1_OFF_W;
    const uint32_t bar0 = sbase + D1_OFF_BAR;
    const uint32_t w_full = bar0, a_full = bar0 + 8, a_empty = bar0 + 16, acc_full = bar0 + 24,
                   acc_empty = bar0 + 32, done = bar0 + 40;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + D1_OFF_MISC);
    volatile int* abort = reinterpret_cast<volatile int*>(smem + D1_OFF_MISC + 4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t n_tiles = (b.n + 127) / 128;
    if (threadIdx.x == 0) {
        *abort = 0;
        mbar_init(w_full, 1);
        mbar_init(a_full, 1);
        mbar_init(a_empty, 1);
        mbar_init(acc_full, 1);
        mbar_init(acc_empty, 128);
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            mbar_expect_tx(w_full, 4 * BW_WCHUNK);
            for (int c = 0; c < 4; ++c) tma_load_2d(sW + c * BW_WCHUNK, &mw2, w_full, 64 * c, 0);
            uint32_t issued = 0;   // A tiles whose loads were issued
            for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
                // the buffer is free once the MMAs of the previous tile completed
                if (issued > 0 && !mbar_wait(a_empty, (issued - 1) & 1u, abort, b.status)) break;
                mbar_expect_tx(a_full, 4 * BW_ATOM);
                for (int q = 0; q < 4; ++q) tma_load_2d(sA + q * BW_ATOM, &mdz2, a_full, 64 * q, (int)(tile * 128));
                ++issued;
            }
            if (*abort) {
                // let the copies still in flight land before the CTA exits
                mbar_drain(w_full, 0);
                if (issued > 0) mbar_drain(a_full, (issued - 1) & 1u);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            bool ok = mbar_wait(w_full, 0, abort, b.status);
            uint32_t it = 0;
            for (int64_t tile = blockIdx.x; ok && tile < n_tiles; tile += gridDim.x, ++it) {
                const uint32_t ph = it & 1u;
                if (!(ok = mbar_wait(a_full, ph, abort, b.status))) break;
                if (it > 0 && !(ok = mbar_wait(acc_empty, (it - 1) & 1u, abort, b.status))) break;
                tc_fence_after();
                for (int c = 0; c < 4; ++c)
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        tc_mma(tmem, sw128_desc(sA + c * BW_ATOM + 32 * kk), sw128_desc(sW + c * BW_WCHUNK + 32 * kk),
                               (c | kk) != 0);
                tc_commit(a_empty);
                tc_commit(acc_full);
            }
            tc_commit(done);
            mbar_drain(done, 0);
        }
    } else {
        const int quarter = warp & 3;
        const int r = 32 * quarter + lane;
        const uint32_t lane_addr = (uint32_t)(32 * quarter) << 16;
        uint32_t it = 0;
        for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++it) {
            if (!__all_sync(0xffffffffu, mbar_wait(acc_full, it & 1u, abort, b.status))) break;
            tc_fence_after();
            const int64_t row = tile * 128 + r;
            const bool live = row < b.n;
#pragma unroll 1
            for (int cc = 0; cc < 8; ++cc) {
                float v[32];
                tc_ld32(tmem + lane_addr + (uint32_t)(32 * cc), v);
                if (!live) continue;
                const float* z = b.Z1 + row * 256 + 32 * cc;
#pragma unroll
                for (int g8 = 0; g8 < 4; ++g8) {
                    const float4 za = *reinterpret_cast<const float4*>(z + 8 * g8);
                    const float4 zb = *reinterpret_cast<const float4*>(z + 8 * g8 + 4);
                    const float zz[8] = {za.x, za.y, za.z, za.w, zb.x, zb.y, zb.z, zb.w};
                    __nv_bfloat16 h[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) h[e] = __float2bfloat16_rn(v[8 * g8 + e] * gelu_grad(zz[e]));
                    const int col = 32 * cc + 8 * g8;
                    *reinterpret_cast<uint4*>(b.dZ1 + row * 256 + col) = *reinterpret_cast<const uint4*>(h);
#pragma unroll
                    for (int e = 0; e < 8; ++e) b.dZ1T[(int64_t)(col + e) * b.ldt + row] = h[e];
                }
            }
            tc_fence_before();
            mbar_arrive(acc_empty);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
    }
}

// --------------------------------------------------------- weight gradients
constexpr int WG_STAGES = 3;
constexpr uint32_t WG_STAGE = BW_ATOM + BW_WCHUNK;   // A [128 x 64] + B [256 x 64]
constexpr uint32_t WG_OFF_BAR = WG_STAGES * WG_STAGE;
constexpr int WG_NBARS = 2 * WG_STAGES + 2;          // full[], empty[], acc_full, done
constexpr uint32_t WG_OFF_MISC = WG_OFF_BAR + 8 * WG_NBARS;
constexpr uint32_t WG_SMEM = WG_OFF_MISC + 16 + 1024;

// item = blockIdx.x: product g (0: dW2 = H1^T dZ2, 1: [dW1; db1] = [X 1]^T
// dZ1), output row tile m (rows 128 m .. 128 m + 127), batch range s; the
// partial goes to part_w[g][s][256][256]
__global__ void __launch_bounds__(BW_THREADS, 1)
    k_mlp_wgrad(const __grid_constant__ CUtensorMap mh1t, const __grid_constant__ CUtensorMap mdz2t,
                const __grid_constant__ CUtensorMap mxt, const __grid_constant__ CUtensorMap mdz1t, BwdArgs b) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar0 = sbase + WG_OFF_BAR;
    auto full = [&](int s) { return bar0 + 8u * s; };
    auto empty = [&](int s) { return bar0 + 8u * (WG_STAGES + s); };
    const uint32_t acc_full = bar0 + 16 * WG_STAGES, done = acc_full + 8;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + WG_OFF_MISC);
    volatile int* abort = reinterpret_cast<volatile int*>(smem + WG_OFF_MISC + 4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = b.splits;
    const int g = blockIdx.x / (2 * S), m = (blockIdx.x / S) % 2, sp = blockIdx.x % S;
    const int64_t k0 = (int64_t)sp * b.split_rows;
    const int64_t k1 = k0 + b.split_rows < b.n ? k0 + b.split_rows : b.n;
    const int nch = k1 > k0 ? (int)((k1 - k0 + 63) / 64) : 0;
    const CUtensorMap* ma = g == 0 ? &mh1t : &mxt;
    const CUtensorMap* mb = g == 0 ? &mdz2t : &mdz1t;
    if (threadIdx.x == 0) {
        *abort = 0;
        for (int s = 0; s < WG_STAGES; ++s) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        mbar_init(acc_full, 1);
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int c = 0;
            for (; c < nch; ++c) {
                const int s = c % WG_STAGES;
                const uint32_t use = (uint32_t)(c / WG_STAGES);
                if (use > 0 && !mbar_wait(empty(s), (use - 1) & 1u, abort, b.status)) break;
                mbar_expect_tx(full(s), WG_STAGE);
                const int x = (int)(k0 + 64 * c);
                tma_load_2d(sbase + s * WG_STAGE, ma, full(s), x, 128 * m);
                tma_load_2d(sbase + s * WG_STAGE + BW_ATOM, mb, full(s), x, 0);
            }
            if (*abort) {
                for (int k = 0; k < WG_STAGES && k < c; ++k) {
                    const int last = c - 1 - k;
                    mbar_drain(full(last % WG_STAGES), (uint32_t)(last / WG_STAGES) & 1u);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            bool ok = true;
            for (int c = 0; c < nch; ++c) {
                const int s = c % WG_STAGES;
                if (!(ok = mbar_wait(full(s), (uint32_t)(c / WG_STAGES) & 1u, abort, b.status))) break;
                tc_fence_after();
                const uint32_t sa = sbase + s * WG_STAGE, sb = sa + BW_ATOM;
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    tc_mma(tmem, sw128_desc(sa + 32 * kk), sw128_desc(sb + 32 * kk), (c | kk) != 0);
                tc_commit(empty(s));
            }
            if (ok) tc_commit(acc_full);
            tc_commit(done);
            mbar_drain(done, 0);
        }
    } else {
        const int quarter = warp & 3;
        const int r = 32 * quarter + lane;
        const uint32_t lane_addr = (uint32_t)(32 * quarter) << 16;
        float* out = b.part_w + (((int64_t)g * S + sp) * 256 + 128 * m + r) * 256;
        const bool have = nch > 0;
        if (!have || __all_sync(0xffffffffu, mbar_wait(acc_full, 0, abort, b.status))) {
            tc_fence_after();
#pragma unroll 1
            for (int cc = 0; cc < 8; ++cc) {
                float v[32];
                if (have) tc_ld32(tmem + lane_addr + (uint32_t)(32 * cc), v);
                else
#pragma unroll
                    for (int j = 0; j < 32; ++j) v[j] = 0.0f;
#pragma unroll
                for (int j = 0; j < 32; j += 4)
                    *reinterpret_cast<float4*>(out + 32 * cc + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
    }
}

// ------------------------------------------------------------------- Adam
// Every gradient the sum of its partials in a fixed order, written to G, then
// one Adam step on the fp32 master parameters; the bf16 copies of w1 and w2
// follow.  Block 0 also sums the loss.
__global__ void k_adam_parts(BwdArgs b, float* p, float* mo, float* ve, float* G, float lr, float b1, float b2,
                             float eps, float c1, float c2, __nv_bfloat16* w1b, __nv_bfloat16* w2b, float* loss) {
    const int S = b.splits;
    const int nbt = (int)((b.n + BT_ROWS - 1) / BT_ROWS);
    const float* pw2 = b.part_w;                            // [S][256][256]
    const float* pw1 = b.part_w + (int64_t)S * 65536;       // [S][256][256], row 192 = b1
    if (blockIdx.x == 0 && threadIdx.x == 0 && loss) {
        float l = 0.0f;
        for (int k = 0; k < nbt; ++k) l += b.part_t[(int64_t)k * BT_PART + 513];
        *loss = l;
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < MLP_NPARAM;
         i += (int64_t)gridDim.x * blockDim.x) {
        float gi = 0.0f;
        if (i < MLP_W1) {
            for (int s = 0; s < S; ++s) gi += pw1[(int64_t)s * 65536 + i];
        } else if (i < MLP_W2_OFF) {
            for (int s = 0; s < S; ++s) gi += pw1[(int64_t)s * 65536 + 192 * 256 + (i - MLP_B1_OFF)];
        } else if (i < MLP_B2_OFF) {
            for (int s = 0; s < S; ++s) gi += pw2[(int64_t)s * 65536 + (i - MLP_W2_OFF)];
        } else if (i < MLP_W3_OFF) {
            for (int k = 0; k < nbt; ++k) gi += b.part_t[(int64_t)k * BT_PART + (i - MLP_B2_OFF)];
        } else if (i < MLP_B3_OFF) {
            for (int k = 0; k < nbt; ++k) gi += b.part_t[(int64_t)k * BT_PART + 256 + (i - MLP_W3_OFF)];
        } else {
            for (int k = 0; k < nbt; ++k) gi += b.part_t[(int64_t)k * BT_PART + 512];
        }
        G[i] = gi;
        const float mi = b1 * mo[i] + (1.0f - b1) * gi;
        const float vi = b2 * ve[i] + (1.0f - b2) * gi * gi;
        mo[i] = mi;
        ve[i] = vi;
        const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        p[i] = pi;
        if (i < MLP_W1) w1b[i] = __float2bfloat16_rn(pi);
        else if (i >= MLP_W2_OFF && i < MLP_W2_OFF + MLP_W2) w2b[i - MLP_W2_OFF] = __float2bfloat16_rn(pi);
    }
}

}  // namespace

int bwd_tail_part_floats(int64_t n) { return (int)((n + BT_ROWS - 1) / BT_ROWS) * BT_PART; }

cudaError_t launch_bwd(const BwdArgs& b, const CUtensorMap& mdz2, const CUtensorMap& mw2, const CUtensorMap& mh1t,
                       const CUtensorMap& mdz2t, const CUtensorMap& mxt, const CUtensorMap& mdz1t, int num_sms,
                       cudaStream_t s) {
    if (b.n <= 0) return cudaSuccess;
    const int64_t nbt = (b.n + BT_ROWS - 1) / BT_ROWS;
    k_bwd_tail<<<(unsigned)nbt, BT_THREADS, 0, s>>>(b);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_mlp_dz1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)D1_SMEM);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (b.n + 127) / 128;
    k_mlp_dz1<<<(unsigned)(tiles < num_sms ? tiles : num_sms), BW_THREADS, D1_SMEM, s>>>(mdz2, mw2, b);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_mlp_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)WG_SMEM);
    if (e != cudaSuccess) return e;
    k_mlp_wgrad<<<(unsigned)(4 * b.splits), BW_THREADS, WG_SMEM, s>>>(mh1t, mdz2t, mxt, mdz1t, b);
    return cudaGetLastError();
}

cudaError_t launch_adam_parts(const BwdArgs& b, float* p, float* m, float* v, float* G, float lr, int step, void* w1b,
                              void* w2b, float* loss, cudaStream_t s) {
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    const int blocks = (int)((MLP_NPARAM + 255) / 256);
    k_adam_parts<<<blocks, 256, 0, s>>>(b, p, m, v, G, lr, b1, b2, 1e-8f, c1, c2, static_cast<__nv_bfloat16*>(w1b),
                                        static_cast<__nv_bfloat16*>(w2b), loss);
    return cudaGetLastError();
}

}  // namespace wh
