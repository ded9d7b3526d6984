// Surrogate kernels for sm_103a: tour features and a small MLP that predicts
// a tour's normalised optimal length (the learned prescreen of local-search
// moves; the paper puts machine learning in the decision loop, Sec. 1 and
// Fig. 1).  MLP 192 -> 256 -> GELU -> 256 -> GELU -> 1, bf16 weights and
// activations, fp32 accumulation; training by forward (k_mlp_tc.cu, on the
// tcgen05 tensor cores), backward and Adam on fp32 master weights, all on the
// device.
//
// The backward GEMMs use the warp-level tensor-core instruction mma.sync
// m16n8k16 (bf16 in, fp32 accumulate) on 128x128x32 shared-memory tiles;
// operands may be transposed, epilogues fuse the GELU derivative or write
// fp32 (the weight gradients in splits of K, reduced in a fixed order).
#include "tour_core.cuh"

namespace wh {

namespace {

constexpr int FEAT_THREADS = 256;
constexpr int G_BM = 128, G_BN = 128, G_BK = 32, G_PAD = 8, G_THREADS = 256;

__device__ __forceinline__ float gelu_grad_f(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// --------------------------------------------------------------- features
// One tour per warp (WarpFeat): lane j gathers the lines of the tour's
// orders j, j + 32, ...; the warp writes the tour's 192 bf16 features.  Row
// r holds tour list[r] when a list is given, else tour r.
__global__ void __launch_bounds__(FEAT_THREADS) k_features(EvalArgs a, FeatConst c, const int32_t* list,
                                                           int64_t n_rows, uint4* X) {
    __shared__ WarpFeat ws[FEAT_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    WarpFeat& w = ws[wid];
    wf_init(w, lane);
    const bool shared_map = a.slot_stride == 0;
    const bool keyed = a.line_key != nullptr;   // per-line keys precomputed (shared slotting)
    const int64_t n_warps = (int64_t)gridDim.x * (FEAT_THREADS / 32);
    for (int64_t r = (int64_t)blockIdx.x * (FEAT_THREADS / 32) + wid; r < n_rows; r += n_warps) {
        const int t = list ? list[r] : (int)r;
        int plan = 0;
        if (!shared_map) {
            int lo = 0, hi = a.n_plans - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (a.plan_tour_off[mid] <= t) lo = mid; else hi = mid - 1;
            }
            plan = lo;
        }
        const int32_t* map = a.slot_map + (int64_t)plan * a.slot_stride;
        const int q0 = a.tour_off[t], q1 = a.tour_off[t + 1];
        bool bad = q0 < 0 || q1 < q0 || (int64_t)q1 > a.n_seq;
        bool over = false;
        uint32_t n_lines = 0;
        for (int qb = q0; !bad && qb < q1; qb += 32) {
            const int q = qb + lane;
            if (q >= q1) continue;
            const int o = a.order_seq[q];
            if ((unsigned)o >= (unsigned)a.n_orders) { bad = true; continue; }
            const int lb = a.order_off[o], le = a.order_off[o + 1];
            if (lb < 0 || le < lb || le > a.n_lines) { bad = true; continue; }
            for (int l = lb; l < le; ++l) {
                uint32_t key;
                if (keyed) {
                    key = a.line_key[l];
                } else {
                    const int s = a.line_sku[l];
                    const int loc = (unsigned)s < (unsigned)a.n_sku ? map[s] : -1;
                    key = (unsigned)loc < (unsigned)a.g.n_loc ? loc_key(a.g, loc) : KEY_BAD;
                }
                if (key == KEY_BAD) { bad = true; break; }
                over |= !wf_insert(w, key);
                ++n_lines;
            }
        }
        bad = __any_sync(0xffffffffu, bad);
        over = __any_sync(0xffffffffu, over);
        n_lines = __reduce_add_sync(0xffffffffu, n_lines);
        if ((bad || over) && lane == 0) flag(a.status, bad ? WH_STATUS_BAD_ORDER : WH_STATUS_TOUR_TOO_LONG);
        wf_finish(w, c, lane, n_lines, X + r * 24);
    }
}

// list <- indices of the set bytes of flag (any order), *count <- their number
__global__ void k_compact_flags(const uint8_t* flag, int64_t n, int32_t* list, int32_t* count) {
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const bool f = i < n && flag[i] != 0;
        const unsigned m = __ballot_sync(0xffffffffu, f);
        int off = 0;
        if (lane == 0 && m) off = atomicAdd(count, __popc(m));
        off = __shfl_sync(0xffffffffu, off, 0);
        if (f) list[off + __popc(m & ((1u << lane) - 1u))] = (int32_t)i;
    }
}

// y_tour[list[j]] = y[j] and clear the tour's flag
__global__ void k_scatter_pred(const int32_t* list, const float* y, int64_t n, float* y_tour, uint8_t* flag) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const int t = list[j];
        y_tour[t] = y[j];
        flag[t] = 0;
    }
}

// ------------------------------------------------------------------ GEMM
enum { EPI_F32 = 1, EPI_GELU_GRAD = 2 };

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C[M,N] = op(A)[M,K] op(B)[K,N]; A(m,k) = transA ? A[k*lda+m] : A[m*lda+k];
// B(k,n) = transB ? B[n*ldb+k] : B[k*ldb+n].  8 warps, 2 x 4 warp grid of
// 64 x 32 warp tiles; fragments per the m16n8k16 layout (row = lane/4,
// k pair = 2*(lane%4)).
template <int EPI>
__global__ void __launch_bounds__(G_THREADS) k_gemm(GemmArgs g) {
    __shared__ __align__(16) __nv_bfloat16 As[G_BM][G_BK + G_PAD];
    __shared__ __align__(16) __nv_bfloat16 Bs[G_BN][G_BK + G_PAD];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 2, wn = warp & 3;
    const int gid = lane >> 2, tig = lane & 3;
    const int64_t m0 = (int64_t)blockIdx.y * G_BM;
    const int n0 = blockIdx.x * G_BN;
    float acc[4][4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.0f;
    const __nv_bfloat16 zero = __float2bfloat16(0.0f);
    // K range of this split (one split unless gridDim.z > 1)
    const int per = (((g.K + (int)gridDim.z - 1) / (int)gridDim.z) + G_BK - 1) / G_BK * G_BK;
    const int k_begin = (int)blockIdx.z * per, k_end = min(g.K, k_begin + per);
    for (int k0 = k_begin; k0 < k_end; k0 += G_BK) {
#pragma unroll 4
        for (int i = 0; i < (G_BM * G_BK) / G_THREADS; ++i) {
            const int e = tid + i * G_THREADS;
            int m, k;
            if (g.transA) { m = e % G_BM; k = e / G_BM; } else { m = e / G_BK; k = e % G_BK; }
            const int64_t gm = m0 + m;
            const int gk = k0 + k;
            __nv_bfloat16 v = zero;
            if (gm < g.M && gk < k_end) v = g.transA ? g.A[(int64_t)gk * g.lda + gm] : g.A[gm * g.lda + gk];
            As[m][k] = v;
        }
#pragma unroll 4
        for (int i = 0; i < (G_BN * G_BK) / G_THREADS; ++i) {
            const int e = tid + i * G_THREADS;
            int n, k;
            if (g.transB) { n = e / G_BK; k = e % G_BK; } else { n = e % G_BN; k = e / G_BN; }
            const int gn = n0 + n, gk = k0 + k;
            __nv_bfloat16 v = zero;
            if (gn < g.N && gk < k_end) v = g.transB ? g.B[(int64_t)gn * g.ldb + gk] : g.B[(int64_t)gk * g.ldb + gn];
            Bs[n][k] = v;
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < G_BK; ks += 16) {
            uint32_t af[4][4], bfr[4][2];
#pragma unroll
            for (int mt = 0; mt < 4; ++mt) {
                const int r = wm * 64 + mt * 16 + gid;
                af[mt][0] = *reinterpret_cast<const uint32_t*>(&As[r][ks + tig * 2]);
                af[mt][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][ks + tig * 2]);
                af[mt][2] = *reinterpret_cast<const uint32_t*>(&As[r][ks + tig * 2 + 8]);
                af[mt][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][ks + tig * 2 + 8]);
            }
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int cidx = wn * 32 + nt * 8 + gid;
                bfr[nt][0] = *reinterpret_cast<const uint32_t*>(&Bs[cidx][ks + tig * 2]);
                bfr[nt][1] = *reinterpret_cast<const uint32_t*>(&Bs[cidx][ks + tig * 2 + 8]);
            }
#pragma unroll
            for (int mt = 0; mt < 4; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) mma_bf16(acc[mt][nt], af[mt], bfr[nt]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int mt = 0; mt < 4; ++mt) {
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int64_t m = m0 + wm * 64 + mt * 16 + gid + (r >= 2 ? 8 : 0);
                const int n = n0 + wn * 32 + nt * 8 + tig * 2 + (r & 1);
                if (m >= g.M || n >= g.N) continue;
                const float v = acc[mt][nt][r];
                if constexpr (EPI == EPI_GELU_GRAD) {
                    g.Cb[m * g.ldc + n] = __float2bfloat16_rn(v * gelu_grad_f(g.Z[m * g.ldz + n]));
                } else if (gridDim.z > 1) {
                    g.Cpart[((int64_t)blockIdx.z * g.M + m) * g.ldc + n] = v;
                } else {
                    g.Cf[m * g.ldc + n] = v;
                }
            }
        }
    }
}

__global__ void k_loss(const float* y, const float* t, int n, float* dy, float* loss) {
    float part = 0.0f;
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x) {
        const float e = y[m] - t[m];
        dy[m] = e / (float)n;
        part += 0.5f * e * e / (float)n;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, part);
}

// dZ2[m,j] = dy[m] * w3[j] * gelu'(Z2[m,j])
__global__ void k_dz2(const float* dy, const float* w3, const float* Z2, int64_t n, __nv_bfloat16* dZ2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n * 256; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = i >> 8;
        const int j = (int)(i & 255);
        dZ2[i] = __float2bfloat16_rn(dy[m] * w3[j] * gelu_grad_f(Z2[i]));
    }
}

// out[j] = sum_m X[m, j] * (scale ? scale[m] : 1), X bf16 [n][cols]; one block per
// 32 columns, threads stride over rows
// column sums of X [n][cols] (rows scaled by scale[m] when given): block
// (x, y) sums columns 32x..32x+31 over the rows of split y; split partials go
// to part[y][cols] (added in order by k_split_reduce), or straight to out
// with one split
__global__ void k_colsum(const __nv_bfloat16* X, int64_t n, int cols, const float* scale, float* out, float* part) {
    __shared__ float ps[8][33];
    const int c = blockIdx.x * 32 + (threadIdx.x & 31);
    const int r0 = threadIdx.x >> 5;
    const int64_t per = (n + gridDim.y - 1) / gridDim.y;
    const int64_t m0 = (int64_t)blockIdx.y * per, m1 = min(n, m0 + per);
    float s = 0.0f;
    if (c < cols)
        for (int64_t m = m0 + r0; m < m1; m += 8) s += __bfloat162float(X[m * cols + c]) * (scale ? scale[m] : 1.0f);
    ps[r0][threadIdx.x & 31] = s;
    __syncthreads();
    if (r0 == 0 && c < cols) {
        float t = 0.0f;
#pragma unroll
        for (int i = 0; i < 8; ++i) t += ps[i][threadIdx.x & 31];
        if (gridDim.y > 1) part[(int64_t)blockIdx.y * cols + c] = t;
        else out[c] = t;
    }
}

__global__ void k_split_reduce(const float* part, int splits, int64_t n, float* out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float t = 0.0f;
        for (int z = 0; z < splits; ++z) t += part[(int64_t)z * n + i];
        out[i] = t;
    }
}

__global__ void k_sum(const float* v, int n, float* out) {
    float s = 0.0f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ float w[32];
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += w[i];
        *out = t;
    }
}

// Adam on fp32 master parameters; refresh the bf16 copies of the GEMM weights
__global__ void k_adam(float* p, float* m, float* v, const float* g, int64_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2, __nv_bfloat16* w1b, __nv_bfloat16* w2b) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        p[i] = pi;
        if (i < MLP_W1) w1b[i] = __float2bfloat16_rn(pi);
        else if (i >= MLP_W2_OFF && i < MLP_W2_OFF + MLP_W2) w2b[i - MLP_W2_OFF] = __float2bfloat16_rn(pi);
    }
}

__global__ void k_to_bf16(const float* p, int64_t n, __nv_bfloat16* out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = __float2bfloat16_rn(p[i]);
}

int blocks_for(int64_t n, int t, int cap = 4096) {
    int64_t b = (n + t - 1) / t;
    if (b > cap) b = cap;
    return b < 1 ? 1 : (int)b;
}

}  // namespace

cudaError_t launch_features(const EvalArgs& a, const FeatConst& c, void* X, const int32_t* list, int64_t n_rows,
                            int num_sms, cudaStream_t s) {
    if (n_rows <= 0) return cudaSuccess;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_features, FEAT_THREADS, 0);
    if (e != cudaSuccess) return e;
    int64_t grid = (int64_t)per_sm * num_sms;
    const int64_t want = (n_rows + FEAT_THREADS / 32 - 1) / (FEAT_THREADS / 32);
    if (grid > want) grid = want;
    if (grid < 1) grid = 1;
    k_features<<<(int)grid, FEAT_THREADS, 0, s>>>(a, c, list, n_rows, static_cast<uint4*>(X));
    return cudaGetLastError();
}

cudaError_t launch_compact_flags(const uint8_t* flag, int64_t n, int32_t* list, int32_t* count, cudaStream_t s) {
    if (cudaMemsetAsync(count, 0, sizeof(int32_t), s) != cudaSuccess) return cudaGetLastError();
    if (n <= 0) return cudaSuccess;
    k_compact_flags<<<blocks_for(n, 256), 256, 0, s>>>(flag, n, list, count);
    return cudaGetLastError();
}

cudaError_t launch_scatter_pred(const int32_t* list, const float* y, int64_t n, float* y_tour, uint8_t* flag,
                                cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_scatter_pred<<<blocks_for(n, 256), 256, 0, s>>>(list, y, n, y_tour, flag);
    return cudaGetLastError();
}

cudaError_t launch_gemm(const GemmArgs& g, int epi, cudaStream_t s) {
    if (g.M <= 0 || g.N <= 0) return cudaSuccess;
    const dim3 grid((g.N + G_BN - 1) / G_BN, (unsigned)((g.M + G_BM - 1) / G_BM));
    if (grid.y > 65535u * 1024u) return cudaErrorInvalidValue;
    if (epi == EPI_GELU_GRAD) k_gemm<EPI_GELU_GRAD><<<grid, G_THREADS, 0, s>>>(g);
    else if (epi == EPI_F32) k_gemm<EPI_F32><<<grid, G_THREADS, 0, s>>>(g);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_train_tail(const float* y, const float* t, int n, float* dy, float* loss, const float* w3,
                              const float* Z2, void* dZ2, cudaStream_t s) {
    k_loss<<<blocks_for(n, 256, 1024), 256, 0, s>>>(y, t, n, dy, loss);
    k_dz2<<<blocks_for((int64_t)n * 256, 256), 256, 0, s>>>(dy, w3, Z2, n, static_cast<__nv_bfloat16*>(dZ2));
    return cudaGetLastError();
}

cudaError_t launch_split_reduce(const float* part, int splits, int64_t n, float* out, cudaStream_t s) {
    k_split_reduce<<<blocks_for(n, 256), 256, 0, s>>>(part, splits, n, out);
    return cudaGetLastError();
}

// split K so that the few output tiles of a weight gradient (K = the batch)
// still fill the GPU; deterministic (fixed-order reduction of the splits)
cudaError_t launch_gemm_splitk(const GemmArgs& g, int splits, cudaStream_t s) {
    if (g.M <= 0 || g.N <= 0) return cudaSuccess;
    if (splits <= 1 || !g.Cpart) return launch_gemm(g, EPI_F32, s);
    const dim3 grid((g.N + G_BN - 1) / G_BN, (unsigned)((g.M + G_BM - 1) / G_BM), (unsigned)splits);
    k_gemm<EPI_F32><<<grid, G_THREADS, 0, s>>>(g);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_split_reduce(g.Cpart, splits, g.M * g.ldc, g.Cf, s);
}

// column sums; the scratch `part` (>= 64 * cols floats) lets the rows split
cudaError_t launch_colsum(const void* X, int64_t n, int cols, const float* scale, float* out, cudaStream_t s,
                          float* part) {
    int splits = part ? (int)((n + 255) / 256) : 1;
    if (splits > 64) splits = 64;
    if (splits < 1) splits = 1;
    k_colsum<<<dim3((cols + 31) / 32, splits), 256, 0, s>>>(static_cast<const __nv_bfloat16*>(X), n, cols, scale,
                                                            out, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || splits == 1) return e;
    return launch_split_reduce(part, splits, cols, out, s);
}

cudaError_t launch_sum(const float* v, int n, float* out, cudaStream_t s) {
    k_sum<<<1, 1024, 0, s>>>(v, n, out);
    return cudaGetLastError();
}

cudaError_t launch_adam(float* p, float* m, float* v, const float* g, int64_t n, float lr, int step, void* w1b,
                        void* w2b, cudaStream_t s) {
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    k_adam<<<blocks_for(n, 256), 256, 0, s>>>(p, m, v, g, n, lr, b1, b2, 1e-8f, c1, c2,
                                              static_cast<__nv_bfloat16*>(w1b), static_cast<__nv_bfloat16*>(w2b));
    return cudaGetLastError();
}

cudaError_t launch_to_bf16(const float* p, int64_t n, void* out, cudaStream_t s) {
    k_to_bf16<<<blocks_for(n, 256), 256, 0, s>>>(p, n, static_cast<__nv_bfloat16*>(out));
    return cudaGetLastError();
}

}  // namespace wh
