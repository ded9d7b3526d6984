// Surrogate kernels for sm_103a: tour features and the helpers of the small
// MLP that predicts a tour's normalised optimal length (the learned prescreen
// of local-search moves; the paper puts machine learning in the decision
// loop, Sec. 1 and Fig. 1).  The MLP's forward (k_mlp_tc.cu) and backward
// (k_mlp_bwd.cu) passes run on the tcgen05 tensor cores; here are the feature
// kernel, the prediction cache's list maintenance and the bf16 copy of the
// parameters.
#include "tour_core.cuh"
#include "feat_core.cuh"

namespace wh {

namespace {

constexpr int FEAT_THREADS = 256;

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

cudaError_t launch_to_bf16(const float* p, int64_t n, void* out, cudaStream_t s) {
    k_to_bf16<<<blocks_for(n, 256), 256, 0, s>>>(p, n, static_cast<__nv_bfloat16*>(out));
    return cudaGetLastError();
}

}  // namespace wh
