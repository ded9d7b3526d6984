// C-ABI of the surrogate MLP (declared in include/wh.h): parameters, Adam
// state and activation scratch on the device; prediction and training steps
// enqueued on the caller's stream.  Forward passes (prediction, and the
// training forward with its saved activations) run the fused tcgen05 kernel
// (k_mlp_tc.cu) on transposed bf16 weights that are refreshed on the stream
// whenever the parameters have changed; the backward runs on the tcgen05
// tensor cores too (k_mlp_bwd.cu), the weight gradients in batch ranges whose
// partials Adam sums in a fixed order.
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
    float* part_w = nullptr;   // [2][kMaxSplits][256][256] weight-gradient partials
    float* part_t = nullptr;   // per 32-row block column sums (b2, w3, b3, loss)
    __nv_bfloat16 *H1 = nullptr, *H2 = nullptr, *dZ2 = nullptr, *dZ1 = nullptr;
    // transposed copies [features][ldt] for the backward's K-major operands
    __nv_bfloat16 *H1T = nullptr, *dZ2T = nullptr, *XT = nullptr, *dZ1T = nullptr;
    __nv_bfloat16 *w1t = nullptr, *w2t = nullptr;   // [256][192], [256][256]: K contiguous
    CUtensorMap mw1, mw2;
    CUtensorMap mw2r;      // w2b [256][256] row-major: the dZ1 product's B operand
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

// 2-D bf16 tensor map of a row-major matrix of `rows` rows whose first
// `cols` elements are read (row stride `ld` elements, a multiple of 8), box
// [box_rows][64] (128 bytes wide, the 128-byte swizzle); elements past the
// ends read as zero
int encode_map_ld(CUtensorMap* m, const void* base, uint64_t rows, uint64_t cols, uint64_t ld, uint32_t box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_tiled();
    if (!fn) return WH_ECUDA;
    const cuuint64_t dim[2] = {cols, rows};
    const cuuint64_t stride[1] = {ld * 2};
    const cuuint32_t box[2] = {64, box_rows};
    const cuuint32_t estride[2] = {1, 1};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dim, stride, box, estride,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? WH_OK : WH_EINVAL;
}

// a dense row-major [rows][cols] matrix
int encode_map(CUtensorMap* m, const void* base, uint64_t rows, uint64_t cols, uint32_t box_rows) {
    return encode_map_ld(m, base, rows, cols, cols, box_rows);
}

// SplitMix64 (Steele, Lea & Flood 2014)
uint64_t sm64(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

void free_all(wh_surrogate* s) {
    void* ptrs[] = {s->P,   s->Mo,  s->Ve,   s->G,   s->w1b,  s->w2b,    s->Z1,     s->Z2,
                    s->y,   s->dy,  s->loss, s->H1,  s->H2,   s->dZ2,    s->dZ1,    s->w1t,
                    s->w2t, s->status, s->part_w, s->part_t, s->H1T, s->dZ2T, s->XT, s->dZ1T};
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

constexpr int kMaxSplits = 16;   // batch ranges of a weight gradient

// rows per batch range of the weight gradients: at least 512, a multiple of
// 64, at most kMaxSplits ranges
int64_t split_rows_for(int64_t n) {
    int64_t r = (n + kMaxSplits - 1) / kMaxSplits;
    r = (r + 63) / 64 * 64;
    return r < 512 ? 512 : r;
}

int64_t ldt_for(int64_t n) { return (n + 63) / 64 * 64; }

int reserve_train(wh_surrogate* s, int64_t n) {
    if (!s->part_w && dalloc(&s->part_w, (size_t)2 * kMaxSplits * 256 * 256)) return WH_ENOMEM;
    if (n <= s->cap) return WH_OK;
    void* old[] = {s->Z1, s->Z2, s->y, s->dy, s->H1, s->H2, s->dZ2, s->dZ1, s->H1T, s->dZ2T, s->XT, s->dZ1T, s->part_t};
    for (void* p : old)
        if (p) cudaFree(p);
    s->Z1 = s->Z2 = s->y = s->dy = s->part_t = nullptr;
    s->H1 = s->H2 = s->dZ2 = s->dZ1 = s->H1T = s->dZ2T = s->XT = s->dZ1T = nullptr;
    s->cap = 0;
    const size_t r = (size_t)n, t = (size_t)ldt_for(n);
    if (dalloc(&s->Z1, r * 256) || dalloc(&s->Z2, r * 256) || dalloc(&s->y, r) || dalloc(&s->dy, r) ||
        dalloc(&s->H1, r * 256) || dalloc(&s->H2, r * 256) || dalloc(&s->dZ2, r * 256) || dalloc(&s->dZ1, r * 256) ||
        dalloc(&s->H1T, 256 * t) || dalloc(&s->dZ2T, 256 * t) || dalloc(&s->XT, 193 * t) ||
        dalloc(&s->dZ1T, 256 * t) || dalloc(&s->part_t, (size_t)wh::bwd_tail_part_floats(n)))
        return WH_ENOMEM;
    s->cap = n;
    return WH_OK;
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
    if (rc == WH_OK) rc = encode_map(&s->mw2r, s->w2b, 256, 256, 256);
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

extern "C" int wh_surrogate_predict_timeout_test(wh_surrogate* s, const uint16_t* X, int64_t n, float* y,
                                                 int64_t skip_tile, uint64_t wait_ns, void* stream) {
    if (!s || n < 1 || !X || !y || skip_tile < 0 || wait_ns < 1000 || wait_ns > 2000000000ull) return WH_EINVAL;
    if (n > kInferChunk || reinterpret_cast<uintptr_t>(X) % 16 != 0) return WH_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = refresh_transposed(s, st);
    if (rc != WH_OK) return rc;
    CUtensorMap mx;
    rc = encode_map(&mx, X, (uint64_t)n, wh::MLP_IN, 128);
    if (rc != WH_OK) return rc;
    if (wh::launch_mlp_tc(mx, s->mw1, s->mw2, s->P, n, y, s->status, s->num_sms, st, nullptr, nullptr, nullptr,
                          nullptr, skip_tile, (unsigned long long)wait_ns) != cudaSuccess)
        return WH_ECUDA;
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
    const int64_t ldt = ldt_for(n);
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
    // backward on the tensor cores: dy, dZ2 and the transposed operands; dZ1;
    // the weight gradients in batch ranges; Adam over their fixed-order sums
    wh::BwdArgs b;
    std::memset(&b, 0, sizeof(b));
    b.n = n;
    b.ldt = ldt;
    b.y = s->y;
    b.t = target;
    b.Z1 = s->Z1;
    b.Z2 = s->Z2;
    b.H1 = s->H1;
    b.H2 = s->H2;
    b.H1T = s->H1T;
    b.X = Xb;
    b.P = s->P;
    b.dy = s->dy;
    b.dZ2 = s->dZ2;
    b.dZ2T = s->dZ2T;
    b.XT = s->XT;
    b.dZ1 = s->dZ1;
    b.dZ1T = s->dZ1T;
    b.part_t = s->part_t;
    b.part_w = s->part_w;
    b.split_rows = split_rows_for(n);
    b.splits = (int32_t)((n + b.split_rows - 1) / b.split_rows);
    b.status = s->status;
    CUtensorMap mdz2, mh1t, mdz2t, mxt, mdz1t;
    rc = encode_map(&mdz2, s->dZ2, (uint64_t)n, 256, 128);
    if (rc == WH_OK) rc = encode_map_ld(&mh1t, s->H1T, 256, (uint64_t)n, (uint64_t)ldt, 128);
    if (rc == WH_OK) rc = encode_map_ld(&mdz2t, s->dZ2T, 256, (uint64_t)n, (uint64_t)ldt, 256);
    if (rc == WH_OK) rc = encode_map_ld(&mxt, s->XT, 193, (uint64_t)n, (uint64_t)ldt, 128);
    if (rc == WH_OK) rc = encode_map_ld(&mdz1t, s->dZ1T, 256, (uint64_t)n, (uint64_t)ldt, 256);
    if (rc != WH_OK) return rc;
    if (wh::launch_bwd(b, mdz2, s->mw2r, mh1t, mdz2t, mxt, mdz1t, s->num_sms, st) != cudaSuccess) return WH_ECUDA;
    s->last_n = n;
    s->step += 1;
    if (wh::launch_adam_parts(b, s->P, s->Mo, s->Ve, s->G, lr, s->step, s->w1b, s->w2b, s->loss, st) != cudaSuccess)
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
