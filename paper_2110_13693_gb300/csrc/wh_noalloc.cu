// wh_eval_plans_noalloc: plan evaluation for callers that cannot allocate
// device memory.
//
// Some callers cannot let a library call cudaMalloc: a serving process whose
// device memory is fully reserved up front by its own pool (an extra
// cudaMalloc would fail or break its memory plan), or code that must never
// trigger the device-wide synchronisation that cudaMalloc / cudaFree can
// cause.  For them this entry point runs the same kernels as wh_eval_plans
// but takes its scratch (per-line keys, the long-tour list, a status word and
// a counter) from one fixed file-scope device array instead of the layout
// handle's cudaMalloc'd buffers.  It needs no handle at all.
//
// The array is part of the library image: every GPU that loads the library
// holds it (about 16 MiB) until the process exits.
#include <cstring>
#include <mutex>

#include "wh_internal.h"

namespace {

constexpr size_t kHeaderBytes = 256;  // [0] status word, [1] long-tour count
constexpr size_t kKeyBytes = sizeof(uint32_t) * (size_t)WH_NOALLOC_MAX_LINES;
constexpr size_t kListBytes = sizeof(int32_t) * 3 * ((size_t)WH_NOALLOC_MAX_TOURS + 1);
constexpr size_t kScratchBytes = kHeaderBytes + kKeyBytes + kListBytes;

// The shared scratch.  Host code must not use this name as a device address:
// in host code it is only a stand-in, so the address is looked up once per
// device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 256;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (looked up on
// the first call made on that device).
int scratch_address(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return WH_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return WH_ERANGE;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return WH_ECUDA;
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return WH_OK;
}

}  // namespace

extern "C" int wh_eval_plans_noalloc(const wh_layout_desc* desc, const wh_orders* orders, const wh_plans* plans,
                                     uint32_t routing_mask, const wh_costs* out, uint32_t* status, void* stream) {
    if (!desc || !orders || !plans || !out) return WH_EINVAL;
    if (routing_mask == 0 || (routing_mask & ~(WH_ROUTE_SSHAPE | WH_ROUTE_OPTIMAL))) return WH_EINVAL;
    const wh_layout_desc d = *desc;
    if (d.n_aisles < 1 || d.slots_per_side < 1 || d.aisle_pitch < 1 || d.slot_pitch < 1 ||
        d.cross_aisle_width < 2 || (d.cross_aisle_width & 1))
        return WH_EINVAL;
    if (d.n_aisles > WH_MAX_AISLES || d.slots_per_side > WH_MAX_SLOTS_PER_SIDE) return WH_ERANGE;
    const int64_t Y = (int64_t)d.cross_aisle_width + (int64_t)(d.slots_per_side - 1) * d.slot_pitch;
    const int64_t span = 2 * (int64_t)(d.n_aisles - 1) * d.aisle_pitch + (int64_t)d.n_aisles * Y;
    if (span >= WH_MAX_TOUR_SPAN) return WH_ERANGE;
    if ((int64_t)d.n_aisles * 2 * d.slots_per_side > 0x7fffffff) return WH_ERANGE;

    const wh_orders o = *orders;
    const wh_plans p = *plans;
    if (o.n_orders < 0 || o.n_lines < 0 || o.n_sku < 0 || p.n_plans < 0 || p.n_tours < 0 || p.n_seq < 0)
        return WH_EINVAL;
    if (p.n_seq > 0x7fffffff) return WH_ERANGE;
    if (o.n_lines > WH_NOALLOC_MAX_LINES || p.n_tours > WH_NOALLOC_MAX_TOURS) return WH_ERANGE;
    if (!o.order_off || (o.n_lines > 0 && !o.line_sku)) return WH_EINVAL;
    if (p.n_plans > 0 && !p.plan_tour_off) return WH_EINVAL;
    if (p.n_tours > 0 && !p.tour_off) return WH_EINVAL;
    if (p.n_seq > 0 && !p.order_seq) return WH_EINVAL;
    if (o.n_lines > 0 && !p.slot_map) return WH_EINVAL;
    if (p.slot_map_stride < 0 || (p.slot_map_stride != 0 && p.slot_map_stride < o.n_sku)) return WH_EINVAL;
    if (p.n_plans == 0) return WH_OK;

    void* base_v = nullptr;
    int rc = scratch_address(&base_v);
    if (rc != WH_OK) return rc;
    unsigned char* base = static_cast<unsigned char*>(base_v);
    int dev = -1, num_sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return WH_ECUDA;
    if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return WH_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    wh::EvalArgs a;
    std::memset(&a, 0, sizeof(a));
    a.g.A = d.n_aisles;
    a.g.L = d.slots_per_side;
    a.g.P = d.aisle_pitch;
    a.g.S = d.slot_pitch;
    a.g.W = d.cross_aisle_width;
    a.g.h = d.cross_aisle_width / 2;
    a.g.Y = (int32_t)Y;
    a.g.n_loc = d.n_aisles * 2 * d.slots_per_side;
    wh::geo_set_div(a.g);
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
    a.max_rec = d.n_aisles < wh::SHORT_MAX ? d.n_aisles : wh::SHORT_MAX;
    // status bits go to the caller's word when given, else to a word inside
    // the array that this call clears and nothing reports
    a.status = status ? status : reinterpret_cast<uint32_t*>(base);
    a.long_count = reinterpret_cast<int32_t*>(base) + 1;
    a.long_cap = p.n_tours;

    wh::Tuning t;
    t.threads = 256;
    t.key16 = 1;
    t.smem_tables = 1;
    if (wh::eval_short_smem_bytes(a, t) > 112 * 1024) t.smem_tables = 0;

    const bool shared_map = p.slot_map_stride == 0;
    uint32_t* line_key = reinterpret_cast<uint32_t*>(base + kHeaderBytes);
    a.line_key = shared_map && o.n_lines > 0 ? line_key : nullptr;
    a.long_list = reinterpret_cast<int32_t*>(base + kHeaderBytes + kKeyBytes);

    // the array keeps the previous call's contents: zero what must start at 0
    // (the status word in use, the caller's or the array's own, here; the
    // long-tour counter in k_prep)
    if (cudaMemsetAsync(a.status, 0, sizeof(uint32_t), s) != cudaSuccess) return WH_ECUDA;
    if (wh::launch_prep(a, s) != cudaSuccess) return WH_ECUDA;
    if (wh::launch_eval_short(a, t, num_sms, s, nullptr) != cudaSuccess) return WH_ECUDA;
    if (p.n_tours > 0) {
        wh::LongArgs L;
        L.single = a;
        L.insts = nullptr;
        L.list = a.long_list;
        L.count = a.long_count;
        L.cap = a.long_cap;
        L.mask = routing_mask;
        if (wh::launch_eval_long(L, shared_map, num_sms, s) != cudaSuccess) return WH_ECUDA;
    }
    return WH_OK;
}
