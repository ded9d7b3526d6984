// C-ABI entry points (declared in include/wh.h): argument checks, the layout
// handle and its device scratch, and the launch sequence of a plan evaluation.
#include <cstring>
#include <new>
#include <vector>

#include "wh_internal.h"

struct wh_layout {
    wh_layout_desc d;
    wh::Geo g;
    int device = -1;
    int num_sms = 0;
    uint32_t* meta = nullptr;     // device: [0] status word, [1] long-tour count
    void* scratch = nullptr;      // device: line keys + long-tour list
    size_t scratch_bytes = 0;
    // kernel timing (wh_set_timing)
    bool timing = false;
    std::vector<cudaEvent_t> events;       // pool, reused across sessions
    std::vector<int> event_kernel;         // kernel id of each recorded pair
    size_t n_recorded = 0;                 // pairs recorded this session
};

namespace {
enum KernelId { K_PREP = 0, K_EVAL_SHORT = 1, K_EVAL_LONG = 2, K_COUNT = 3 };
const char* const kKernelNames[K_COUNT] = {"k_prep", "k_eval_short", "k_eval_long"};

// Brackets one launch with events when timing is on.
class LaunchTimer {
  public:
    LaunchTimer(wh_layout* h, int kernel, cudaStream_t s) : h_(h), s_(s) {
        if (!h_->timing) return;
        const size_t need = 2 * (h_->n_recorded + 1);
        while (h_->events.size() < need) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) { ok_ = false; return; }
            h_->events.push_back(e);
        }
        if (h_->event_kernel.size() < h_->n_recorded + 1) h_->event_kernel.resize(h_->n_recorded + 1);
        h_->event_kernel[h_->n_recorded] = kernel;
        ok_ = cudaEventRecord(h_->events[2 * h_->n_recorded], s_) == cudaSuccess;
        armed_ = ok_;
    }
    ~LaunchTimer() {
        if (!armed_) return;
        if (cudaEventRecord(h_->events[2 * h_->n_recorded + 1], s_) == cudaSuccess) ++h_->n_recorded;
    }
    bool ok() const { return ok_; }

  private:
    wh_layout* h_;
    cudaStream_t s_;
    bool ok_ = true;
    bool armed_ = false;
};
}  // namespace

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

class DeviceGuard {
  public:
    explicit DeviceGuard(int dev) {
        if (dev >= 0 && cudaGetDevice(&prev_) == cudaSuccess && prev_ != dev) {
            if (cudaSetDevice(dev) == cudaSuccess) switched_ = true;
        }
    }
    ~DeviceGuard() {
        if (switched_) cudaSetDevice(prev_);
    }

  private:
    int prev_ = -1;
    bool switched_ = false;
};

// Bind the handle to the current device on first use; later calls must run on
// the same device.
int bind_device(wh_layout* h) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return WH_ECUDA;
    if (h->device == dev) return WH_OK;
    if (h->device != -1) return WH_EINVAL;
    if (cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return WH_ECUDA;
    void* p = nullptr;
    if (cudaMalloc(&p, kAlign) != cudaSuccess) return WH_ENOMEM;
    if (cudaMemset(p, 0, kAlign) != cudaSuccess) {
        cudaFree(p);
        return WH_ECUDA;
    }
    h->meta = static_cast<uint32_t*>(p);
    h->device = dev;
    return WH_OK;
}

int reserve_scratch(wh_layout* h, size_t bytes) {
    if (bytes <= h->scratch_bytes) return WH_OK;
    if (h->scratch) {
        cudaFree(h->scratch);  // synchronises the device before releasing
        h->scratch = nullptr;
        h->scratch_bytes = 0;
    }
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return WH_ENOMEM;
    }
    h->scratch = p;
    h->scratch_bytes = bytes;
    return WH_OK;
}

wh::Tuning default_tuning(const wh::EvalArgs& a) {
    wh::Tuning t;
    t.threads = 256;
    t.key16 = 1;
    t.smem_tables = 1;
    // keep two 256-thread CTAs per SM; larger order books stay in global memory
    if (wh::eval_short_smem_bytes(a, t) > 112 * 1024) t.smem_tables = 0;
    return t;
}

}  // namespace

extern "C" int wh_create_layout(const wh_layout_desc* desc, wh_layout** out) {
    if (!desc || !out) return WH_EINVAL;
    const wh_layout_desc d = *desc;
    if (d.n_aisles < 1 || d.slots_per_side < 1 || d.aisle_pitch < 1 || d.slot_pitch < 1 ||
        d.cross_aisle_width < 2 || (d.cross_aisle_width & 1))
        return WH_EINVAL;
    if (d.n_aisles > WH_MAX_AISLES || d.slots_per_side > WH_MAX_SLOTS_PER_SIDE) return WH_ERANGE;
    const int64_t Y = (int64_t)d.cross_aisle_width + (int64_t)(d.slots_per_side - 1) * d.slot_pitch;
    const int64_t span = 2 * (int64_t)(d.n_aisles - 1) * d.aisle_pitch + (int64_t)d.n_aisles * Y;
    if (span >= WH_MAX_TOUR_SPAN) return WH_ERANGE;
    if ((int64_t)d.n_aisles * 2 * d.slots_per_side > 0x7fffffff) return WH_ERANGE;
    wh_layout* h = new (std::nothrow) wh_layout;
    if (!h) return WH_ENOMEM;
    h->d = d;
    h->g.A = d.n_aisles;
    h->g.L = d.slots_per_side;
    h->g.P = d.aisle_pitch;
    h->g.S = d.slot_pitch;
    h->g.W = d.cross_aisle_width;
    h->g.h = d.cross_aisle_width / 2;
    h->g.Y = (int32_t)Y;
    h->g.n_loc = d.n_aisles * 2 * d.slots_per_side;
    *out = h;
    return WH_OK;
}

extern "C" int wh_eval_plans(wh_layout* h, const wh_orders* orders, const wh_plans* plans, uint32_t routing_mask,
                             const wh_costs* out, void* stream) {
    if (!h || !orders || !plans || !out) return WH_EINVAL;
    if (routing_mask == 0 || (routing_mask & ~(WH_ROUTE_SSHAPE | WH_ROUTE_OPTIMAL))) return WH_EINVAL;
    const wh_orders o = *orders;
    const wh_plans p = *plans;
    if (o.n_orders < 0 || o.n_lines < 0 || o.n_sku < 0 || p.n_plans < 0 || p.n_tours < 0 || p.n_seq < 0)
        return WH_EINVAL;
    if (p.n_seq > 0x7fffffff) return WH_ERANGE;
    if (!o.order_off || (o.n_lines > 0 && !o.line_sku)) return WH_EINVAL;
    if (p.n_plans > 0 && !p.plan_tour_off) return WH_EINVAL;
    if (p.n_tours > 0 && !p.tour_off) return WH_EINVAL;
    if (p.n_seq > 0 && !p.order_seq) return WH_EINVAL;
    if (o.n_lines > 0 && !p.slot_map) return WH_EINVAL;
    if (p.slot_map_stride < 0 || (p.slot_map_stride != 0 && p.slot_map_stride < o.n_sku)) return WH_EINVAL;
    if (p.n_plans == 0) return WH_OK;

    int rc = bind_device(h);
    if (rc != WH_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    wh::EvalArgs a;
    std::memset(&a, 0, sizeof(a));
    a.g = h->g;
    a.n_orders = o.n_orders;
    a.n_lines = o.n_lines;
    a.n_sku = o.n_sku;
    a.order_off = o.order_off;
    a.line_sku = o.line_sku;
    a.slot_map = p.slot_map;
    a.slot_stride = p.slot_map_stride;
    a.n_plans = p.n_plans;
    a.n_tours = p.n_tours;
    a.n_seq = p.n_seq;
    a.plan_tour_off = p.plan_tour_off;
    a.tour_off = p.tour_off;
    a.order_seq = p.order_seq;
    a.tour_s = out->tour_s;
    a.tour_rr = out->tour_rr;
    a.plan_s = out->plan_s;
    a.plan_rr = out->plan_rr;
    a.mask = routing_mask;
    a.max_rec = h->g.A < wh::SHORT_MAX ? h->g.A : wh::SHORT_MAX;
    a.status = h->meta;
    a.long_count = reinterpret_cast<int32_t*>(h->meta + 1);

    const wh::Tuning t = default_tuning(a);

    const bool shared_map = p.slot_map_stride == 0;
    const size_t key_bytes = shared_map ? align_up(sizeof(uint32_t) * (size_t)o.n_lines) : 0;
    const size_t list_bytes = align_up(sizeof(int32_t) * 2 * ((size_t)p.n_tours + 1));
    rc = reserve_scratch(h, key_bytes + list_bytes);
    if (rc != WH_OK) return rc;
    char* base = static_cast<char*>(h->scratch);
    uint32_t* line_key = shared_map && o.n_lines > 0 ? reinterpret_cast<uint32_t*>(base) : nullptr;
    a.line_key = line_key;
    a.long_list = reinterpret_cast<int32_t*>(base + key_bytes);

    {
        LaunchTimer lt(h, K_PREP, s);
        if (!lt.ok() || wh::launch_prep(a, line_key, s) != cudaSuccess) return WH_ECUDA;
    }
    {
        LaunchTimer lt(h, K_EVAL_SHORT, s);
        if (!lt.ok() || wh::launch_eval_short(a, t, h->num_sms, s, nullptr) != cudaSuccess) return WH_ECUDA;
    }
    if (p.n_tours > 0) {
        LaunchTimer lt(h, K_EVAL_LONG, s);
        if (!lt.ok() || wh::launch_eval_long(a, h->num_sms, s) != cudaSuccess) return WH_ECUDA;
    }
    return WH_OK;
}

extern "C" int wh_get_last_status(wh_layout* h, void* stream, uint32_t* status) {
    if (!h || !status) return WH_EINVAL;
    if (h->device < 0) {
        *status = 0;
        return WH_OK;
    }
    DeviceGuard guard(h->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t v = 0;
    if (cudaMemcpyAsync(&v, h->meta, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess) return WH_ECUDA;
    if (cudaMemsetAsync(h->meta, 0, sizeof(uint32_t), s) != cudaSuccess) return WH_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return WH_ECUDA;
    *status = v;
    return WH_OK;
}

extern "C" int wh_set_timing(wh_layout* h, int enable) {
    if (!h) return WH_EINVAL;
    h->timing = enable != 0;
    h->n_recorded = 0;
    return WH_OK;
}

extern "C" int wh_get_timing(wh_layout* h, int32_t* n_kernels, const char** names, int32_t* launches,
                             double* total_ms, int32_t cap) {
    if (!h || !n_kernels || cap < 0 || (cap > 0 && (!names || !launches || !total_ms))) return WH_EINVAL;
    double ms[K_COUNT] = {0, 0, 0};
    int32_t cnt[K_COUNT] = {0, 0, 0};
    if (h->n_recorded > 0) {
        DeviceGuard guard(h->device);
        for (size_t i = 0; i < h->n_recorded; ++i) {
            float e = 0.f;
            if (cudaEventSynchronize(h->events[2 * i + 1]) != cudaSuccess) return WH_ECUDA;
            if (cudaEventElapsedTime(&e, h->events[2 * i], h->events[2 * i + 1]) != cudaSuccess) return WH_ECUDA;
            ms[h->event_kernel[i]] += e;
            cnt[h->event_kernel[i]] += 1;
        }
    }
    *n_kernels = K_COUNT;
    for (int32_t k = 0; k < K_COUNT && k < cap; ++k) {
        names[k] = kKernelNames[k];
        launches[k] = cnt[k];
        total_ms[k] = ms[k];
    }
    return WH_OK;
}

extern "C" void wh_destroy(wh_layout* h) {
    if (!h) return;
    if (h->device >= 0) {
        DeviceGuard guard(h->device);
        for (cudaEvent_t e : h->events) cudaEventDestroy(e);
        if (h->scratch) cudaFree(h->scratch);
        if (h->meta) cudaFree(h->meta);
    }
    delete h;
}
