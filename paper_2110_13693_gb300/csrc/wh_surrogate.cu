// C-ABI of the surrogate MLP (declared in include/wh.h): parameters, Adam
// state and activation scratch on the device; prediction and training steps
// enqueued on the caller's stream.  Forward passes (prediction, and the
// training forward with its saved activations) run the fused tcgen05 kernel
// (k_mlp_tc.cu) on transposed bf16 weights that are refreshed on the stream
// whenever the parameters have changed; the backward GEMMs run on mma.sync
// (k_surrogate.cu), the weight gradients split along the batch.
#include <cudaTypedefs.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "wh_internal.h"

struct wh_surrogate {
    int device = -1;
    float* P = nullptr;    // fp32 master parameters [MLP_NPARAM]
    float* Mo = nullptr;   // Adam first moment
    float* Ve = nullptr;   // Adam second moment
    float* G = nullptr;    // last gradients
    __nv_bfloat16* w1b = nullptr;
    __nv_bfloat16* w2b = nullptr;
    int step = 0;
    int64_t cap = 0;       // rows of training scratch
    int64_t last_n = 0;    // rows of the last training step (its saved intermediates)
    float *Z1 = nullptr, *Z2 = nullptr, *y = nullptr, *dy = nullptr, *loss = nullptr;
    float* part = nullptr; // split partials of the weight gradients and column sums
    __nv_bfloat16 *H1 = nullptr, *H2 = nullptr, *dZ2 = nullptr, *dZ1 = nullptr;
    __nv_bfloat16 *w1t = nullptr, *w2t = nullptr;   // [256][192], [256][256]: K contiguous
    CUtensorMap mw1, mw2;
    bool t_stale = true;   // w1t / w2t lag the parameters
    int* status = nullptr; // WH_STATUS_* bits of the inference kernel
    int num_sms = 0;
};

namespace {

// rows per inference launch: TMA row coordinates are 32-bit
constexpr int64_t kInferChunk = (int64_t)1 << 30;

PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// 2-D bf16 tensor map of a row-major [rows][cols] matrix, box [box_rows][64]
// (128 bytes wide, the 128-byte swizzle), rows past the end read as zero
int encode_map(CUtensorMap* m, const void* base, uint64_t rows, uint64_t cols, uint32_t box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_tiled();
    if (!fn) return WH_ECUDA;
    const cuuint64_t dim[2] = {cols, rows};
    const cuuint64_t stride[1] = {cols * 2};
    const cuuint32_t box[2] = {64, box_rows};
    const cuuint32_t estride[2] = {1, 1};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dim, stride, box, estride,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? WH_OK : WH_EINVAL;
}

// SplitMix64 (Steele, Lea & Flood 2014)
uint64_t sm64(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

void free_all(wh_surrogate* s) {
    void* ptrs[] = {s->P, s->Mo, s->Ve, s->G, s->w1b, s->w2b, s->Z1, s->Z2, s->y, s->dy, s->loss,
                    s->H1, s->H2, s->dZ2, s->dZ1, s->w1t, s->w2t, s->status, s->part};
    for (void* p : ptrs)
        if (p) cudaFree(p);
}

int upload_params(wh_surrogate* s, const float* host) {
    if (cudaMemcpy(s->P, host, sizeof(float) * wh::MLP_NPARAM, cudaMemcpyHostToDevice) != cudaSuccess) return WH_ECUDA;
    if (wh::launch_to_bf16(s->P, wh::MLP_W1, s->w1b, nullptr) != cudaSuccess) return WH_ECUDA;
    if (wh::launch_to_bf16(s->P + wh::MLP_W2_OFF, wh::MLP_W2, s->w2b, nullptr) != cudaSuccess) return WH_ECUDA;
    s->t_stale = true;
    return cudaDeviceSynchronize() == cudaSuccess ? WH_OK : WH_ECUDA;
}

template <typename T>
int dalloc(T** p, size_t n) {
    if (cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (n ? n : 1)) != cudaSuccess) {
        cudaGetLastError();
        return WH_ENOMEM;
    }
    return WH_OK;
}

constexpr int kMaxSplits = 32;   // K splits of a weight gradient (K = the batch)

int splits_for(int64_t n) {
    const int64_t k = (n + 127) / 128;
    return (int)(k < 1 ? 1 : (k > kMaxSplits ? kMaxSplits : k));
}

int reserve_train(wh_surrogate* s, int64_t n) {
    if (!s->part && dalloc(&s->part, (size_t)kMaxSplits * 256 * 256)) return WH_ENOMEM;
    if (n <= s->cap) return WH_OK;
    void* old[] = {s->Z1, s->Z2, s->y, s->dy, s->H1, s->H2, s->dZ2, s->dZ1};
    for (void* p : old)
        if (p) cudaFree(p);
    s->cap = 0;
    const size_t r = (size_t)n;
    if (dalloc(&s->Z1, r * 256) || dalloc(&s->Z2, r * 256) || dalloc(&s->y, r) || dalloc(&s->dy, r) ||
        dalloc(&s->H1, r * 256) || dalloc(&s->H2, r * 256) || dalloc(&s->dZ2, r * 256) || dalloc(&s->dZ1, r * 256))
        return WH_ENOMEM;
    s->cap = n;
    return WH_OK;
}

wh::GemmArgs gemm(int64_t M, int N, int K, const __nv_bfloat16* A, int64_t lda, int ta, const __nv_bfloat16* B,
                  int64_t ldb, int tb) {
    wh::GemmArgs g;
    std::memset(&g, 0, sizeof(g));
    g.M = M;
    g.N = N;
    g.K = K;
    g.A = A;
    g.lda = lda;
    g.transA = ta;
    g.B = B;
    g.ldb = ldb;
    g.transB = tb;
    return g;
}

// the transposed bf16 weights the tensor maps describe, when stale
int refresh_transposed(wh_surrogate* s, cudaStream_t st) {
    if (!s->t_stale) return WH_OK;
    if (wh::launch_transpose_bf16(s->P, 192, 256, s->w1t, st) != cudaSuccess ||
        wh::launch_transpose_bf16(s->P + wh::MLP_W2_OFF, 256, 256, s->w2t, st) != cudaSuccess)
        return WH_ECUDA;
    s->t_stale = false;
    return WH_OK;
}

}  // namespace

extern "C" int wh_surrogate_create(uint64_t seed, wh_surrogate** out) {
    if (!out) return WH_EINVAL;
    wh_surrogate* s = new (std::nothrow) wh_surrogate;
    if (!s) return WH_ENOMEM;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return WH_ECUDA;
    }
    if (dalloc(&s->P, wh::MLP_NPARAM) || dalloc(&s->Mo, wh::MLP_NPARAM) || dalloc(&s->Ve, wh::MLP_NPARAM) ||
        dalloc(&s->G, wh::MLP_NPARAM) || dalloc(&s->w1b, wh::MLP_W1) || dalloc(&s->w2b, wh::MLP_W2) ||
        dalloc(&s->loss, 1) || dalloc(&s->w1t, wh::MLP_W1) || dalloc(&s->w2t, wh::MLP_W2) || dalloc(&s->status, 1)) {
        free_all(s);
        delete s;
        return WH_ENOMEM;
    }
    // Xavier-uniform weights, zero biases
    std::vector<float> h(wh::MLP_NPARAM, 0.0f);
    uint64_t st = seed ^ 0x6A09E667F3BCC909ull;
    auto fill = [&](int64_t off, int64_t n, int fan_in, int fan_out) {
        const double bound = std::sqrt(6.0 / (fan_in + fan_out));
        for (int64_t i = 0; i < n; ++i) {
            const double u = (double)(sm64(st) >> 11) * (1.0 / 9007199254740992.0);
            h[off + i] = (float)((2.0 * u - 1.0) * bound);
        }
    };
    fill(0, wh::MLP_W1, 192, 256);
    fill(wh::MLP_W2_OFF, wh::MLP_W2, 256, 256);
    fill(wh::MLP_W3_OFF, 256, 256, 1);
    int rc = cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device) == cudaSuccess ? WH_OK
                                                                                                         : WH_ECUDA;
    if (rc == WH_OK) rc = encode_map(&s->mw1, s->w1t, 256, 192, 256);
    if (rc == WH_OK) rc = encode_map(&s->mw2, s->w2t, 256, 256, 256);
    if (rc == WH_OK) rc = upload_params(s, h.data());
    if (rc == WH_OK && (cudaMemset(s->status, 0, sizeof(int)) != cudaSuccess ||
                        cudaMemset(s->Mo, 0, sizeof(float) * wh::MLP_NPARAM) != cudaSuccess ||
                        cudaMemset(s->Ve, 0, sizeof(float) * wh::MLP_NPARAM) != cudaSuccess ||
                        cudaMemset(s->G, 0, sizeof(float) * wh::MLP_NPARAM) != cudaSuccess))
        rc = WH_ECUDA;
    if (rc != WH_OK) {
        free_all(s);
        delete s;
        return rc;
    }
    *out = s;
    return WH_OK;
}

extern "C" int wh_surrogate_set_params(wh_surrogate* s, const float* host_params) {
    if (!s || !host_params) return WH_EINVAL;
    int rc = upload_params(s, host_params);
    if (rc != WH_OK) return rc;
    s->step = 0;
    if (cudaMemset(s->Mo, 0, sizeof(float) * wh::MLP_NPARAM) != cudaSuccess ||
        cudaMemset(s->Ve, 0, sizeof(float) * wh::MLP_NPARAM) != cudaSuccess)
        return WH_ECUDA;
    return WH_OK;
}

extern "C" int wh_surrogate_get_params(wh_surrogate* s, float* host_params, float* host_grads) {
    if (!s || (!host_params && !host_grads)) return WH_EINVAL;
    if (cudaDeviceSynchronize() != cudaSuccess) return WH_ECUDA;
    if (host_params &&
        cudaMemcpy(host_params, s->P, sizeof(float) * wh::MLP_NPARAM, cudaMemcpyDeviceToHost) != cudaSuccess)
        return WH_ECUDA;
    if (host_grads && cudaMemcpy(host_grads, s->G, sizeof(float) * wh::MLP_NPARAM, cudaMemcpyDeviceToHost) != cudaSuccess)
        return WH_ECUDA;
    return WH_OK;
}

extern "C" int wh_surrogate_predict(wh_surrogate* s, const uint16_t* X, int64_t n, float* y, void* stream) {
    if (!s || n < 0 || (n > 0 && (!X || !y))) return WH_EINVAL;
    if (n == 0) return WH_OK;
    if (reinterpret_cast<uintptr_t>(X) % 16 != 0) return WH_EINVAL;   // TMA base alignment
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc0 = refresh_transposed(s, st);
    if (rc0 != WH_OK) return rc0;
    for (int64_t r = 0; r < n; r += kInferChunk) {
        const int64_t m = n - r < kInferChunk ? n - r : kInferChunk;
        CUtensorMap mx;
        int rc = encode_map(&mx, X + r * wh::MLP_IN, (uint64_t)m, wh::MLP_IN, 128);
        if (rc != WH_OK) return rc;
        if (wh::launch_mlp_tc(mx, s->mw1, s->mw2, s->P, m, y + r, s->status, s->num_sms, st) != cudaSuccess)
            return WH_ECUDA;
    }
    return WH_OK;
}

extern "C" int wh_surrogate_get_status(wh_surrogate* s, uint32_t* out) {
    if (!s || !out) return WH_EINVAL;
    int v = 0;
    if (cudaMemcpy(&v, s->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return WH_ECUDA;
    if (cudaMemset(s->status, 0, sizeof(int)) != cudaSuccess) return WH_ECUDA;
    *out = (uint32_t)v;
    return WH_OK;
}

extern "C" int wh_surrogate_train_step(wh_surrogate* s, const uint16_t* X, const float* target, int32_t n, float lr,
                                       float* loss_out, void* stream) {
    if (!s || n < 1 || !X || !target || !(lr > 0.0f)) return WH_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = reserve_train(s, n);
    if (rc != WH_OK) return rc;
    const __nv_bfloat16* Xb = reinterpret_cast<const __nv_bfloat16*>(X);
    // forward on the tensor cores, keeping both layers' pre-activations and
    // activations for the backward pass
    if (reinterpret_cast<uintptr_t>(X) % 16 != 0) return WH_EINVAL;
    rc = refresh_transposed(s, st);
    if (rc != WH_OK) return rc;
    {
        CUtensorMap mx;
        rc = encode_map(&mx, X, (uint64_t)n, wh::MLP_IN, 128);
        if (rc != WH_OK) return rc;
        if (wh::launch_mlp_tc(mx, s->mw1, s->mw2, s->P, n, s->y, s->status, s->num_sms, st, s->Z1, s->H1, s->Z2,
                              s->H2) != cudaSuccess)
            return WH_ECUDA;
    }
    if (cudaMemsetAsync(s->loss, 0, sizeof(float), st) != cudaSuccess) return WH_ECUDA;
    if (wh::launch_train_tail(s->y, target, n, s->dy, s->loss, s->P + wh::MLP_W3_OFF, s->Z2, s->dZ2, st) !=
        cudaSuccess)
        return WH_ECUDA;
    // output layer
    if (wh::launch_colsum(s->H2, n, 256, s->dy, s->G + wh::MLP_W3_OFF, st, s->part) != cudaSuccess) return WH_ECUDA;
    if (wh::launch_sum(s->dy, n, s->G + wh::MLP_B3_OFF, st) != cudaSuccess) return WH_ECUDA;
    // layer 2: dW2 = H1^T dZ2, db2 = colsum dZ2, dZ1 = (dZ2 W2^T) * gelu'(Z1)
    if (wh::launch_colsum(s->dZ2, n, 256, nullptr, s->G + wh::MLP_B2_OFF, st, s->part) != cudaSuccess)
        return WH_ECUDA;
    wh::GemmArgs gw2 = gemm(256, 256, n, s->H1, 256, 1, s->dZ2, 256, 0);
    gw2.Cpart = s->part;
    gw2.Cf = s->G + wh::MLP_W2_OFF;
    gw2.ldc = 256;
    if (wh::launch_gemm_splitk(gw2, splits_for(n), st) != cudaSuccess) return WH_ECUDA;
    wh::GemmArgs gd1 = gemm(n, 256, 256, s->dZ2, 256, 0, s->w2b, 256, 1);
    gd1.Z = s->Z1;
    gd1.ldz = 256;
    gd1.Cb = s->dZ1;
    gd1.ldc = 256;
    if (wh::launch_gemm(gd1, 2, st) != cudaSuccess) return WH_ECUDA;
    // layer 1: dW1 = X^T dZ1, db1 = colsum dZ1
    if (wh::launch_colsum(s->dZ1, n, 256, nullptr, s->G + wh::MLP_B1_OFF, st, s->part) != cudaSuccess)
        return WH_ECUDA;
    wh::GemmArgs gw1 = gemm(192, 256, n, Xb, 192, 1, s->dZ1, 256, 0);
    gw1.Cpart = s->part;
    gw1.Cf = s->G;
    gw1.ldc = 256;
    if (wh::launch_gemm_splitk(gw1, splits_for(n), st) != cudaSuccess) return WH_ECUDA;
    s->last_n = n;
    s->step += 1;
    if (wh::launch_adam(s->P, s->Mo, s->Ve, s->G, wh::MLP_NPARAM, lr, s->step, s->w1b, s->w2b, st) != cudaSuccess)
        return WH_ECUDA;
    s->t_stale = true;
    if (loss_out && cudaMemcpyAsync(loss_out, s->loss, sizeof(float), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return WH_ECUDA;
    return WH_OK;
}

extern "C" int wh_surrogate_get_trace(wh_surrogate* s, int32_t which, void* dst, int64_t n_rows, void* stream) {
    if (!s || !dst || n_rows < 0 || n_rows > s->last_n) return WH_EINVAL;
    const void* src = nullptr;
    size_t row_bytes = 0;
    switch (which) {
        case WH_TRACE_Z1: src = s->Z1; row_bytes = 256 * sizeof(float); break;
        case WH_TRACE_H1: src = s->H1; row_bytes = 256 * sizeof(__nv_bfloat16); break;
        case WH_TRACE_Z2: src = s->Z2; row_bytes = 256 * sizeof(float); break;
        case WH_TRACE_H2: src = s->H2; row_bytes = 256 * sizeof(__nv_bfloat16); break;
        case WH_TRACE_Y: src = s->y; row_bytes = sizeof(float); break;
        case WH_TRACE_DY: src = s->dy; row_bytes = sizeof(float); break;
        case WH_TRACE_DZ2: src = s->dZ2; row_bytes = 256 * sizeof(__nv_bfloat16); break;
        case WH_TRACE_DZ1: src = s->dZ1; row_bytes = 256 * sizeof(__nv_bfloat16); break;
        default: return WH_EINVAL;
    }
    if (n_rows == 0) return WH_OK;
    if (cudaMemcpyAsync(dst, src, row_bytes * (size_t)n_rows, cudaMemcpyDeviceToDevice,
                        static_cast<cudaStream_t>(stream)) != cudaSuccess)
        return WH_ECUDA;
    return WH_OK;
}

extern "C" void wh_surrogate_destroy(wh_surrogate* s) {
    if (!s) return;
    free_all(s);
    delete s;
}
