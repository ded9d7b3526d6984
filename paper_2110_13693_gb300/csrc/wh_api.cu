// C-ABI entry points (declared in include/wh.h): argument checks, the layout
// handle and its device scratch, the launch sequence of a plan evaluation, the
// batched persistent launch with CUDA-graph replay, and its autotuner.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>
#include <iterator>

#include "wh_internal.h"

// Per-kernel CUDA-event timing of a handle's launches (wh_set_timing,
// wh_batch_set_timing): a pool of event pairs, reused across sessions.
struct KernelTiming {
    bool on = false;
    std::vector<cudaEvent_t> events;       // pairs: [2i] before, [2i+1] after launch i
    std::vector<int> kernel;               // kernel id of each recorded pair
    size_t n = 0;                          // pairs recorded this session
};

struct wh_layout {
    wh_layout_desc d;
    wh::Geo g;
    int device = -1;
    int num_sms = 0;
    uint32_t* meta = nullptr;     // device: [0] status word, [1] long-tour count
    void* scratch = nullptr;      // device: line keys + long-tour list
    size_t scratch_bytes = 0;
    void* mv_scratch = nullptr;   // device: move-evaluation index structures
    size_t mv_scratch_bytes = 0;
    void* mv_tasks = nullptr;     // device: move tasks + their costs + long-task list
    size_t mv_tasks_bytes = 0;
    void* mv_long = nullptr;      // device: long tasks' record matrix, record counts, largest keys
    size_t mv_long_bytes = 0;
    void* sr_scratch = nullptr;   // device: screening features and predictions
    size_t sr_scratch_bytes = 0;
    // the task list of the last wh_eval_moves call (for wh_ls_apply's cost update)
    const int32_t* last_moves = nullptr;
    int32_t last_n_moves = 0;
    const int64_t* last_task_off = nullptr;
    const int4* last_tasks = nullptr;
    const int2* last_task_cost = nullptr;
    // the last wh_surrogate_screen call's task list, counted flags and rows
    int64_t screen_n_tasks = 0;
    const int4* screen_tasks = nullptr;
    const int2* screen_counted = nullptr;
    const uint16_t* screen_rows = nullptr;
    KernelTiming timing;                   // wh_set_timing
};

struct wh_batch {
    int device = -1;
    int num_sms = 0;
    int32_t n_inst = 0;
    std::vector<wh::EvalArgs> args;        // host copy of the per-instance descriptors
    wh::EvalArgs* d_args = nullptr;
    wh::WorkItem* d_items = nullptr;
    int32_t n_items = 0;
    size_t items_cap = 0;
    uint32_t* meta = nullptr;              // [0] status, [1] long count, [2] queue
    void* scratch = nullptr;               // line keys of all instances + long list + long records
    uint2* long_rec = nullptr;             // the long-tour kernel's record scratch (in scratch)
    bool key16 = true;
    bool id16 = false;   // the instances' order ids are 16-bit
    int32_t max_orders = 0, max_lines = 0, max_rec = 0, max_work = 0;
    int64_t total_tours = 0;
    int32_t long_cap = 0;
    wh::Tuning tune{};
    int32_t chunks_per_item = 16;
    cudaStream_t capture = nullptr;
    cudaGraphExec_t graphs[4] = {nullptr, nullptr, nullptr, nullptr};   // per routing mask
    KernelTiming timing;                   // wh_batch_set_timing (eager launches only)
};

namespace {
enum KernelId { K_PREP = 0, K_EVAL_SHORT = 1, K_EVAL_LONG = 2, K_EVAL_SSHAPE = 3, K_COUNT = 4 };
const char* const kKernelNames[K_COUNT] = {"k_prep", "k_eval_short", "k_eval_long", "k_eval_sshape"};

// Brackets one launch with events when timing is on.
class LaunchTimer {
  public:
    LaunchTimer(KernelTiming& t, int kernel, cudaStream_t s) : t_(t), s_(s) {
        if (!t_.on) return;
        const size_t need = 2 * (t_.n + 1);
        while (t_.events.size() < need) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) { ok_ = false; return; }
            t_.events.push_back(e);
        }
        if (t_.kernel.size() < t_.n + 1) t_.kernel.resize(t_.n + 1);
        t_.kernel[t_.n] = kernel;
        ok_ = cudaEventRecord(t_.events[2 * t_.n], s_) == cudaSuccess;
        armed_ = ok_;
    }
    ~LaunchTimer() {
        if (!armed_) return;
        if (cudaEventRecord(t_.events[2 * t_.n + 1], s_) == cudaSuccess) ++t_.n;
    }
    bool ok() const { return ok_; }

  private:
    KernelTiming& t_;
    cudaStream_t s_;
    bool ok_ = true;
    bool armed_ = false;
};

// Per-kernel launches and summed milliseconds of a timing session
// (synchronises on the recorded events).
int read_timing(const KernelTiming& t, int n_kinds, const char* const* kinds, int32_t* n_kernels,
                const char** names, int32_t* launches, double* total_ms, int32_t cap) {
    std::vector<double> ms(n_kinds, 0.0);
    std::vector<int32_t> cnt(n_kinds, 0);
    for (size_t i = 0; i < t.n; ++i) {
        float e = 0.f;
        if (cudaEventSynchronize(t.events[2 * i + 1]) != cudaSuccess) return WH_ECUDA;
        if (cudaEventElapsedTime(&e, t.events[2 * i], t.events[2 * i + 1]) != cudaSuccess) return WH_ECUDA;
        ms[t.kernel[i]] += e;
        cnt[t.kernel[i]] += 1;
    }
    *n_kernels = n_kinds;
    for (int32_t k = 0; k < n_kinds && k < cap; ++k) {
        names[k] = kinds[k];
        launches[k] = cnt[k];
        total_ms[k] = ms[k];
    }
    return WH_OK;
}

void free_timing(KernelTiming& t) {
    for (cudaEvent_t e : t.events) cudaEventDestroy(e);
    t.events.clear();
}

constexpr size_t kAlign = 256;
constexpr int32_t kBatchLongCap = 1 << 22;

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

int check_desc(const wh_layout_desc& d, wh::Geo* g) {
    if (d.n_aisles < 1 || d.slots_per_side < 1 || d.aisle_pitch < 1 || d.slot_pitch < 1 ||
        d.cross_aisle_width < 2 || (d.cross_aisle_width & 1))
        return WH_EINVAL;
    if (d.n_aisles > WH_MAX_AISLES || d.slots_per_side > WH_MAX_SLOTS_PER_SIDE) return WH_ERANGE;
    const int64_t Y = (int64_t)d.cross_aisle_width + (int64_t)(d.slots_per_side - 1) * d.slot_pitch;
    const int64_t span = 2 * (int64_t)(d.n_aisles - 1) * d.aisle_pitch + (int64_t)d.n_aisles * Y;
    if (span >= WH_MAX_TOUR_SPAN) return WH_ERANGE;
    if ((int64_t)d.n_aisles * 2 * d.slots_per_side > 0x7fffffff) return WH_ERANGE;
    g->A = d.n_aisles;
    g->L = d.slots_per_side;
    g->P = d.aisle_pitch;
    g->S = d.slot_pitch;
    g->W = d.cross_aisle_width;
    g->h = d.cross_aisle_width / 2;
    g->Y = (int32_t)Y;
    g->n_loc = d.n_aisles * 2 * d.slots_per_side;
    wh::geo_set_div(*g);
    return WH_OK;
}

int check_problem(const wh_orders& o, const wh_plans& p) {
    if (o.n_orders < 0 || o.n_lines < 0 || o.n_sku < 0 || p.n_plans < 0 || p.n_tours < 0 || p.n_seq < 0)
        return WH_EINVAL;
    if (p.n_seq > 0x7fffffff) return WH_ERANGE;
    if (!o.order_off || (o.n_lines > 0 && !o.line_sku)) return WH_EINVAL;
    if (p.n_plans > 0 && !p.plan_tour_off) return WH_EINVAL;
    if (p.n_tours > 0 && !p.tour_off) return WH_EINVAL;
    if (p.n_seq > 0 && !p.order_seq) return WH_EINVAL;
    if (o.n_lines > 0 && !p.slot_map) return WH_EINVAL;
    if (p.slot_map_stride < 0 || (p.slot_map_stride != 0 && p.slot_map_stride < o.n_sku)) return WH_EINVAL;
    return WH_OK;
}

void fill_args(wh::EvalArgs& a, const wh::Geo& g, const wh_orders& o, const wh_plans& p, const wh_costs& out,
               uint32_t mask) {
    std::memset(&a, 0, sizeof(a));
    a.g = g;
    a.n_orders = o.n_orders;
    a.n_lines = o.n_lines;
    a.n_sku = o.n_sku;
    a.order_off = o.order_off;
    a.line_sku = o.line_sku;
    a.slot_map = p.slot_map;
    a.slot_stride = p.slot_map_stride;
    a.loc_used = p.loc_used;
    a.n_plans = p.n_plans;
    a.n_tours = p.n_tours;
    a.n_seq = p.n_seq;
    a.plan_tour_off = p.plan_tour_off;
    a.tour_off = p.tour_off;
    a.order_seq = p.order_seq;
    a.tour_s = out.tour_s;
    a.tour_rr = out.tour_rr;
    a.plan_s = out.plan_s;
    a.plan_rr = out.plan_rr;
    a.mask = mask;
    // record slots per thread: a tour of more pick aisles goes to the
    // long-tour pass (rare: a tour of <= 64 lines rarely visits more than 32
    // aisles), so the per-thread buffers stay at 32 slots
    a.max_rec = g.A < wh::SHORT_MAX / 2 ? g.A : wh::SHORT_MAX / 2;
}

int device_info(int* dev, int* sms) {
    if (cudaGetDevice(dev) != cudaSuccess) return WH_ECUDA;
    if (cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, *dev) != cudaSuccess) return WH_ECUDA;
    return WH_OK;
}

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

int grow(void** buf, size_t* have, size_t bytes) {
    if (bytes <= *have) return WH_OK;
    if (*buf) {
        cudaFree(*buf);  // synchronises the device before releasing
        *buf = nullptr;
        *have = 0;
    }
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return WH_ENOMEM;
    }
    *buf = p;
    *have = bytes;
    return WH_OK;
}

int reserve_scratch(wh_layout* h, size_t bytes) { return grow(&h->scratch, &h->scratch_bytes, bytes); }

wh::Tuning default_tuning(const wh::EvalArgs& a) {
    wh::Tuning t;
    t.key16 = 1;
    t.threads = wh::key16_ok(a.g) ? 384 : 256;
    t.smem_tables = 1;
    // keep two CTAs per SM; larger order books stay in global memory
    if (wh::eval_short_smem_bytes(a, t) > 112 * 1024) t.smem_tables = 0;
    return t;
}

}  // namespace

extern "C" int wh_create_layout(const wh_layout_desc* desc, wh_layout** out) {
    if (!desc || !out) return WH_EINVAL;
    wh::Geo g;
    const int rc = check_desc(*desc, &g);
    if (rc != WH_OK) return rc;
    wh_layout* h = new (std::nothrow) wh_layout;
    if (!h) return WH_ENOMEM;
    h->d = *desc;
    h->g = g;
    *out = h;
    return WH_OK;
}

extern "C" int wh_eval_plans(wh_layout* h, const wh_orders* orders, const wh_plans* plans, uint32_t routing_mask,
                             const wh_costs* out, void* stream) {
    if (!h || !orders || !plans || !out) return WH_EINVAL;
    if (routing_mask == 0 || (routing_mask & ~(WH_ROUTE_SSHAPE | WH_ROUTE_OPTIMAL))) return WH_EINVAL;
    const wh_orders o = *orders;
    const wh_plans p = *plans;
    int rc = check_problem(o, p);
    if (rc != WH_OK) return rc;
    if (p.n_plans == 0) return WH_OK;

    rc = bind_device(h);
    if (rc != WH_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    wh::EvalArgs a;
    fill_args(a, h->g, o, p, *out, routing_mask);
    a.status = h->meta;
    a.long_count = reinterpret_cast<int32_t*>(h->meta + 1);
    a.long_cap = p.n_tours;
    const wh::Tuning t = default_tuning(a);

    const bool shared_map = p.slot_map_stride == 0;
    // S-shape alone under a shared slotting on <= 64 aisles: per-order
    // aggregates instead of per-line keys
    const bool agg = shared_map && routing_mask == WH_ROUTE_SSHAPE && h->g.A <= 64 && o.n_orders > 0;
    const size_t key_bytes = shared_map && !agg ? align_up(sizeof(uint32_t) * (size_t)o.n_lines) : 0;
    const size_t agg_bytes = agg ? align_up(sizeof(uint4) * (size_t)o.n_orders) : 0;
    const size_t list_bytes = align_up(sizeof(int32_t) * 3 * ((size_t)p.n_tours + 1));
    const size_t rec_bytes = align_up(wh::long_rec_bytes(h->num_sms));
    rc = reserve_scratch(h, key_bytes + agg_bytes + list_bytes + rec_bytes);
    if (rc != WH_OK) return rc;
    char* base = static_cast<char*>(h->scratch);
    a.line_key = shared_map && !agg && o.n_lines > 0 ? reinterpret_cast<uint32_t*>(base) : nullptr;
    a.order_agg = agg ? reinterpret_cast<uint4*>(base + key_bytes) : nullptr;
    a.long_list = reinterpret_cast<int32_t*>(base + key_bytes + agg_bytes);
    uint2* long_rec = rec_bytes ? reinterpret_cast<uint2*>(base + key_bytes + agg_bytes + list_bytes) : nullptr;

    {
        LaunchTimer lt(h->timing, K_PREP, s);
        if (!lt.ok() || wh::launch_prep(a, s) != cudaSuccess) return WH_ECUDA;
    }
    {
        LaunchTimer lt(h->timing, wh::sshape_kernel_applies(a) ? K_EVAL_SSHAPE : K_EVAL_SHORT, s);
        if (!lt.ok() || wh::launch_eval_short(a, t, h->num_sms, s, nullptr) != cudaSuccess) return WH_ECUDA;
    }
    // the S-shape-only kernels keep every tour in its thread: no long-tour pass
    if (p.n_tours > 0 && !wh::sshape_kernel_applies(a)) {
        LaunchTimer lt(h->timing, K_EVAL_LONG, s);
        wh::LongArgs L;
        L.single = a;
        L.insts = nullptr;
        L.list = a.long_list;
        L.count = a.long_count;
        L.cap = a.long_cap;
        L.mask = routing_mask;
        L.rec = long_rec;
        if (!lt.ok() || wh::launch_eval_long(L, shared_map, h->num_sms, s) != cudaSuccess) return WH_ECUDA;
    }
    return WH_OK;
}

namespace {

// Scratch, index structures and the task list of a move evaluation (up to
// and including the task fill).  Synchronises `s` once to size the list.
// reuse_index: the order -> tour table, tour line counts and SKU -> orders
// index that the previous preparation on this handle built for the same
// plans and order book are used as they are (within one call only).
int prepare_moves(wh_layout* h, const wh_orders& o, const wh_plans& p, const int32_t* moves, int32_t n_moves,
                  int32_t max_orders, int32_t max_lines, int64_t* delta, int32_t* status, wh::MoveArgs& M,
                  cudaStream_t s, bool reuse_index = false) {
    // the scratch is about to be reused: the last screen's trace goes stale
    h->screen_n_tasks = 0;
    h->screen_tasks = nullptr;
    h->screen_counted = nullptr;
    h->screen_rows = nullptr;
    std::memset(&M, 0, sizeof(M));
    wh_costs none;
    std::memset(&none, 0, sizeof(none));
    fill_args(M.a, h->g, o, p, none, WH_ROUTE_SSHAPE | WH_ROUTE_OPTIMAL);
    M.a.status = h->meta;
    M.moves = reinterpret_cast<const int4*>(moves);
    M.n_moves = n_moves;
    M.max_orders = max_orders;
    M.max_lines = max_lines;
    M.delta = delta;
    M.mstatus = status;
    M.long_count = reinterpret_cast<int32_t*>(h->meta + 2);
    M.stats = reinterpret_cast<unsigned long long*>(h->meta + 4);

    const size_t n_ot = (size_t)p.n_plans * (size_t)o.n_orders;
    const size_t nb = ((size_t)n_moves + 1 + 1023) / 1024;
    size_t off[7], total = 0;
    const size_t sizes[7] = {sizeof(int32_t) * n_ot, sizeof(int32_t) * ((size_t)p.n_tours + 1),
                             sizeof(int32_t) * ((size_t)o.n_sku + 1), sizeof(int32_t) * ((size_t)o.n_sku + 1),
                             sizeof(int32_t) * ((size_t)o.n_lines + 1), sizeof(int64_t) * ((size_t)n_moves + 1),
                             sizeof(int64_t) * (nb + 1)};
    for (int i = 0; i < 7; ++i) {
        off[i] = total;
        total += align_up(sizes[i]);
    }
    // reusing the index: the previous preparation's buffers must stay where
    // they are (the kept set is never larger than the screened one)
    if (reuse_index && total > h->mv_scratch_bytes) return WH_EINVAL;
    int rc = grow(&h->mv_scratch, &h->mv_scratch_bytes, total);
    if (rc != WH_OK) return rc;
    char* base = static_cast<char*>(h->mv_scratch);
    M.order_tour = reinterpret_cast<int32_t*>(base + off[0]);
    M.tour_lines = reinterpret_cast<int32_t*>(base + off[1]);
    M.sku_off = reinterpret_cast<int32_t*>(base + off[2]);
    M.sku_cur = reinterpret_cast<int32_t*>(base + off[3]);
    M.sku_orders = reinterpret_cast<int32_t*>(base + off[4]);
    M.task_off = reinterpret_cast<int64_t*>(base + off[5]);
    M.scan_aux = reinterpret_cast<int64_t*>(base + off[6]);

    if (wh::launch_moves_prepare(M, h->num_sms, s, reuse_index) != cudaSuccess) return WH_ECUDA;
    int64_t n_tasks = 0;
    if (cudaMemcpyAsync(&n_tasks, M.task_off + n_moves, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return WH_ECUDA;
    if (n_tasks < 0 || n_tasks > ((int64_t)1 << 40)) return WH_ECUDA;
    M.n_tasks = n_tasks;
    M.long_cap = (int32_t)std::min<int64_t>(n_tasks + 1, 0x7fffffff);
    const size_t task_bytes = align_up(sizeof(int4) * (size_t)(n_tasks + 1));
    const size_t cost_bytes = align_up(sizeof(int2) * (size_t)(n_tasks + 1));
    rc = grow(&h->mv_tasks, &h->mv_tasks_bytes, task_bytes + cost_bytes + align_up(sizeof(int32_t) * (size_t)M.long_cap));
    if (rc != WH_OK) return rc;
    char* tb = static_cast<char*>(h->mv_tasks);
    M.tasks = reinterpret_cast<int4*>(tb);
    M.task_cost = reinterpret_cast<int2*>(tb + task_bytes);
    M.long_list = reinterpret_cast<int32_t*>(tb + task_bytes + cost_bytes);
    return WH_OK;
}

}  // namespace

namespace {

// The long tasks listed by the short-task pass: read their number (one
// stream synchronisation), size the record matrix, run the record and DP
// kernels, then the final status pass.
int eval_long_tasks(wh_layout* h, wh::MoveArgs& M, cudaStream_t s) {
    int32_t n_long = 0;
    if (M.n_tasks > 0) {
        if (cudaMemcpyAsync(&n_long, M.long_count, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return WH_ECUDA;
        n_long = std::min(n_long, M.long_cap);
    }
    M.long_rec_cap = n_long;
    if (n_long > 0) {
        const size_t rec = align_up(sizeof(uint2) * (size_t)wh::MVL_RMAX * (size_t)n_long);
        const size_t col = align_up(sizeof(int32_t) * (size_t)n_long);
        const int rc = grow(&h->mv_long, &h->mv_long_bytes, rec + 2 * col);
        if (rc != WH_OK) return rc;
        char* b = static_cast<char*>(h->mv_long);
        M.long_rec = reinterpret_cast<uint2*>(b);
        M.long_m = reinterpret_cast<int32_t*>(b + rec);
        M.long_key = reinterpret_cast<uint32_t*>(b + rec + col);
    }
    return wh::launch_moves_long(M, h->num_sms, s) == cudaSuccess ? WH_OK : WH_ECUDA;
}

}  // namespace

extern "C" int wh_eval_moves(wh_layout* h, const wh_orders* orders, const wh_plans* plans, const int32_t* tour_s,
                             const int32_t* tour_rr, const int32_t* moves, int32_t n_moves, int32_t max_orders,
                             int32_t max_lines, int64_t* delta, int32_t* status, void* stream) {
    if (!h || !orders || !plans || n_moves < 0 || max_orders < 0 || max_lines < 0) return WH_EINVAL;
    const wh_orders o = *orders;
    const wh_plans p = *plans;
    int rc = check_problem(o, p);
    if (rc != WH_OK) return rc;
    if (n_moves == 0) return WH_OK;
    if (!moves || !delta || !status || !tour_s || !tour_rr || p.n_plans < 1) return WH_EINVAL;
    rc = bind_device(h);
    if (rc != WH_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    h->last_moves = nullptr;
    wh::MoveArgs M;
    rc = prepare_moves(h, o, p, moves, n_moves, max_orders, max_lines, delta, status, M, s);
    if (rc != WH_OK) return rc;
    M.tour_s_old = tour_s;
    M.tour_rr_old = tour_rr;
    const bool k16 = wh::key16_ok(h->g);
    if (wh::launch_moves_eval(M, k16, h->num_sms, s) != cudaSuccess) return WH_ECUDA;
    rc = eval_long_tasks(h, M, s);
    if (rc != WH_OK) return rc;
    h->last_moves = moves;
    h->last_n_moves = n_moves;
    h->last_task_off = M.task_off;
    h->last_tasks = M.tasks;
    h->last_task_cost = M.task_cost;
    return WH_OK;
}

namespace {

// The prescreen of wh_surrogate_screen after its argument checks (n_plans >= 1,
// device bound): index, task list, features, predictions, selection.
int screen_moves(wh_layout* h, wh_surrogate* sg, const wh_orders& o, const wh_plans& p, const int32_t* moves,
                 int32_t moves_per_plan, int32_t keep, int32_t max_orders, int32_t max_lines, float* y_tour_cache,
                 uint8_t* tour_changed, int32_t* kept, void* stream) {
    const int32_t n_moves = (int32_t)((int64_t)p.n_plans * moves_per_plan);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc = WH_OK;
    h->last_moves = nullptr;
    // per-move status and the task list (into the screening scratch's delta/status)
    const size_t feat_row = sizeof(uint16_t) * WH_FEATURES;
    wh::MoveArgs M;
    // status, delta and scores live in the screening scratch
    const size_t head = align_up(sizeof(int32_t) * (size_t)n_moves) + align_up(sizeof(int64_t) * 2 * (size_t)n_moves) +
                        align_up(sizeof(float) * (size_t)n_moves);
    rc = grow(&h->sr_scratch, &h->sr_scratch_bytes, head);
    if (rc != WH_OK) return rc;
    {
        char* b = static_cast<char*>(h->sr_scratch);
        int32_t* st = reinterpret_cast<int32_t*>(b);
        int64_t* dl = reinterpret_cast<int64_t*>(b + align_up(sizeof(int32_t) * (size_t)n_moves));
        rc = prepare_moves(h, o, p, moves, n_moves, max_orders, max_lines, dl, st, M, s);
        if (rc != WH_OK) return rc;
    }
    if (wh::launch_moves_fill(M, s) != cudaSuccess) return WH_ECUDA;
    // features and predictions of the current tours and of the tasks' changed tours
    const size_t need = head + align_up(feat_row * (size_t)(p.n_tours + 1)) + align_up(sizeof(float) * (size_t)(p.n_tours + 1)) +
                        align_up(feat_row * (size_t)(M.n_tasks + 1)) + align_up(sizeof(float) * (size_t)(M.n_tasks + 1)) +
                        align_up(sizeof(int32_t) * (size_t)(p.n_tours + 2));
    if (need > h->sr_scratch_bytes) {
        // grow keeping nothing: the head (status, delta) must be rebuilt, so
        // size for the worst case and redo the preparation
        rc = grow(&h->sr_scratch, &h->sr_scratch_bytes, need + need / 4);
        if (rc != WH_OK) return rc;
        char* b = static_cast<char*>(h->sr_scratch);
        int32_t* st = reinterpret_cast<int32_t*>(b);
        int64_t* dl = reinterpret_cast<int64_t*>(b + align_up(sizeof(int32_t) * (size_t)n_moves));
        rc = prepare_moves(h, o, p, moves, n_moves, max_orders, max_lines, dl, st, M, s);
        if (rc != WH_OK) return rc;
        if (wh::launch_moves_fill(M, s) != cudaSuccess) return WH_ECUDA;
    }
    char* b = static_cast<char*>(h->sr_scratch);
    size_t at = align_up(sizeof(int32_t) * (size_t)n_moves) + align_up(sizeof(int64_t) * 2 * (size_t)n_moves);
    float* score = reinterpret_cast<float*>(b + at);
    at = head;
    uint16_t* X_tour = reinterpret_cast<uint16_t*>(b + at);
    at += align_up(feat_row * (size_t)(p.n_tours + 1));
    float* y_tour = reinterpret_cast<float*>(b + at);
    at += align_up(sizeof(float) * (size_t)(p.n_tours + 1));
    uint16_t* X_task = reinterpret_cast<uint16_t*>(b + at);
    at += align_up(feat_row * (size_t)(M.n_tasks + 1));
    float* y_task = reinterpret_cast<float*>(b + at);
    at += align_up(sizeof(float) * (size_t)(M.n_tasks + 1));
    int32_t* list = reinterpret_cast<int32_t*>(b + at);   // [n_tours] + count

    wh::FeatConst c;
    c.A = h->g.A;
    c.L = h->g.L;
    c.magic_a = (((uint64_t)1 << 40) + (uint64_t)h->g.A - 1) / (uint64_t)h->g.A;
    c.magic_l = (((uint64_t)1 << 40) + (uint64_t)h->g.L - 1) / (uint64_t)h->g.L;
    c.inv_a = (float)(1.0 / (double)h->g.A);
    // predictions of the current tours: all of them, or (with a cache) the
    // flagged ones, scattered into the cache
    if (!tour_changed) {
        float* yt = y_tour_cache ? y_tour_cache : y_tour;
        if (wh::launch_features(M.a, c, X_tour, nullptr, p.n_tours, h->num_sms, s) != cudaSuccess) return WH_ECUDA;
        rc = wh_surrogate_predict(sg, X_tour, p.n_tours, yt, stream);
        if (rc != WH_OK) return rc;
    } else {
        int32_t* count = list + p.n_tours + 1;
        if (wh::launch_compact_flags(tour_changed, p.n_tours, list, count, s) != cudaSuccess) return WH_ECUDA;
        int32_t n_changed = 0;
        if (cudaMemcpyAsync(&n_changed, count, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return WH_ECUDA;
        if (n_changed > 0) {
            if (wh::launch_features(M.a, c, X_tour, list, n_changed, h->num_sms, s) != cudaSuccess) return WH_ECUDA;
            rc = wh_surrogate_predict(sg, X_tour, n_changed, y_tour, stream);
            if (rc != WH_OK) return rc;
            if (wh::launch_scatter_pred(list, y_tour, n_changed, y_tour_cache, tour_changed, s) != cudaSuccess)
                return WH_ECUDA;
        }
    }
    if (wh::launch_task_features(M, c, X_task, h->num_sms, s) != cudaSuccess) return WH_ECUDA;
    h->screen_n_tasks = M.n_tasks;
    h->screen_tasks = M.tasks;
    h->screen_counted = M.task_cost;
    h->screen_rows = X_task;
    rc = wh_surrogate_predict(sg, X_task, M.n_tasks, y_task, stream);
    if (rc != WH_OK) return rc;
    wh::ScreenArgs S;
    S.M = M;
    S.y_tour = y_tour_cache ? y_tour_cache : y_tour;
    S.y_task = y_task;
    S.score = score;
    S.moves_per_plan = moves_per_plan;
    S.keep = keep;
    S.kept = reinterpret_cast<int4*>(kept);
    return wh::launch_screen_select(S, s) == cudaSuccess ? WH_OK : WH_ECUDA;
}

int screen_args_ok(wh_layout* h, wh_surrogate* sg, const wh_orders* orders, const wh_plans* plans,
                   const int32_t* moves, int32_t moves_per_plan, int32_t keep, int32_t max_orders, int32_t max_lines,
                   const float* y_tour_cache, const uint8_t* tour_changed, const int32_t* kept) {
    if (!h || !sg || !orders || !plans || !moves || !kept || moves_per_plan < 1 || moves_per_plan > 256 ||
        keep < 1 || keep > moves_per_plan || max_orders < 0 || max_lines < 0 || (tour_changed && !y_tour_cache))
        return WH_EINVAL;
    int rc = check_problem(*orders, *plans);
    if (rc != WH_OK) return rc;
    if (h->g.L > 256) return WH_ERANGE;
    if ((int64_t)plans->n_plans * moves_per_plan > 0x7fffffff) return WH_ERANGE;
    return WH_OK;
}

}  // namespace

extern "C" int wh_surrogate_screen(wh_layout* h, wh_surrogate* sg, const wh_orders* orders, const wh_plans* plans,
                                   const int32_t* moves, int32_t moves_per_plan, int32_t keep, int32_t max_orders,
                                   int32_t max_lines, float* y_tour_cache, uint8_t* tour_changed, int32_t* kept,
                                   void* stream) {
    int rc = screen_args_ok(h, sg, orders, plans, moves, moves_per_plan, keep, max_orders, max_lines, y_tour_cache,
                            tour_changed, kept);
    if (rc != WH_OK) return rc;
    if (plans->n_plans == 0) return WH_OK;
    rc = bind_device(h);
    if (rc != WH_OK) return rc;
    return screen_moves(h, sg, *orders, *plans, moves, moves_per_plan, keep, max_orders, max_lines, y_tour_cache,
                        tour_changed, kept, stream);
}

extern "C" int wh_surrogate_screen_eval(wh_layout* h, wh_surrogate* sg, const wh_orders* orders,
                                        const wh_plans* plans, const int32_t* moves, int32_t moves_per_plan,
                                        int32_t keep, int32_t max_orders, int32_t max_lines, float* y_tour_cache,
                                        uint8_t* tour_changed, const int32_t* tour_s, const int32_t* tour_rr,
                                        int32_t* kept, int64_t* kept_delta, int32_t* kept_status, void* stream) {
    int rc = screen_args_ok(h, sg, orders, plans, moves, moves_per_plan, keep, max_orders, max_lines, y_tour_cache,
                            tour_changed, kept);
    if (rc != WH_OK) return rc;
    if (plans->n_plans == 0) return WH_OK;
    if (!tour_s || !tour_rr || !kept_delta || !kept_status) return WH_EINVAL;
    rc = bind_device(h);
    if (rc != WH_OK) return rc;
    rc = screen_moves(h, sg, *orders, *plans, moves, moves_per_plan, keep, max_orders, max_lines, y_tour_cache,
                      tour_changed, kept, stream);
    if (rc != WH_OK) return rc;
    // the kept moves scored exactly on the prescreen's index (the same plans):
    // checks, task counts, task list, short and long tasks
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int32_t n_kept = plans->n_plans * keep;
    wh::MoveArgs M;
    rc = prepare_moves(h, *orders, *plans, kept, n_kept, max_orders, max_lines, kept_delta, kept_status, M, s, true);
    if (rc != WH_OK) return rc;
    M.tour_s_old = tour_s;
    M.tour_rr_old = tour_rr;
    if (wh::launch_moves_eval(M, wh::key16_ok(h->g), h->num_sms, s) != cudaSuccess) return WH_ECUDA;
    rc = eval_long_tasks(h, M, s);
    if (rc != WH_OK) return rc;
    h->last_moves = kept;
    h->last_n_moves = n_kept;
    h->last_task_off = M.task_off;
    h->last_tasks = M.tasks;
    h->last_task_cost = M.task_cost;
    return WH_OK;
}

extern "C" int wh_surrogate_screen_trace(wh_layout* h, int64_t* n_tasks, const int32_t** tasks, const int32_t** counted,
                                         const uint16_t** features) {
    if (!h || !n_tasks || !tasks || !counted || !features) return WH_EINVAL;
    *n_tasks = h->screen_n_tasks;
    *tasks = reinterpret_cast<const int32_t*>(h->screen_tasks);
    *counted = reinterpret_cast<const int32_t*>(h->screen_counted);
    *features = h->screen_rows;
    return WH_OK;
}

extern "C" int wh_ls_apply(wh_layout* h, const wh_orders* orders, const wh_plans* plans, const int32_t* moves,
                           int32_t moves_per_plan, const int64_t* delta, const int32_t* status, int32_t* applied,
                           const wh_costs* costs, uint8_t* tour_changed, void* stream) {
    if (!h || !orders || !plans || moves_per_plan < 1 || moves_per_plan > 256) return WH_EINVAL;
    const wh_orders o = *orders;
    const wh_plans p = *plans;
    int rc = check_problem(o, p);
    if (rc != WH_OK) return rc;
    if (p.n_plans == 0) return WH_OK;
    if (!moves || !delta || !status || !applied || (tour_changed && !costs)) return WH_EINVAL;
    if (o.n_orders > 50000) return WH_ERANGE;
    rc = bind_device(h);
    if (rc != WH_OK) return rc;
    wh::LsArgs L;
    std::memset(&L, 0, sizeof(L));
    wh_costs none;
    std::memset(&none, 0, sizeof(none));
    fill_args(L.a, h->g, o, p, none, WH_ROUTE_OPTIMAL);
    L.a.status = h->meta;
    L.moves = reinterpret_cast<const int4*>(moves);
    L.moves_per_plan = moves_per_plan;
    L.delta = delta;
    L.status = status;
    L.applied = applied;
    L.seg_cap = std::max(o.n_orders, 1);
    if (costs) {
        if (h->last_moves != moves || (int64_t)h->last_n_moves != (int64_t)p.n_plans * moves_per_plan) return WH_EINVAL;
        L.task_off = h->last_task_off;
        L.tasks = h->last_tasks;
        L.task_cost = h->last_task_cost;
        L.tour_s = costs->tour_s;
        L.tour_rr = costs->tour_rr;
        L.plan_s = costs->plan_s;
        L.plan_rr = costs->plan_rr;
        L.tour_changed = tour_changed;
    }
    return wh::launch_ls_apply(L, static_cast<cudaStream_t>(stream)) == cudaSuccess ? WH_OK : WH_ECUDA;
}

extern "C" int wh_surrogate_features(wh_layout* h, const wh_orders* orders, const wh_plans* plans, uint16_t* X,
                                     void* stream) {
    if (!h || !orders || !plans) return WH_EINVAL;
    const wh_orders o = *orders;
    const wh_plans p = *plans;
    int rc = check_problem(o, p);
    if (rc != WH_OK) return rc;
    if (h->g.L > 256) return WH_ERANGE;
    if (p.n_plans == 0 || p.n_tours == 0) return WH_OK;
    if (!X) return WH_EINVAL;
    rc = bind_device(h);
    if (rc != WH_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    wh::EvalArgs a;
    wh_costs none;
    std::memset(&none, 0, sizeof(none));
    fill_args(a, h->g, o, p, none, WH_ROUTE_OPTIMAL);
    a.status = h->meta;
    a.long_count = reinterpret_cast<int32_t*>(h->meta + 1);
    const bool shared_map = p.slot_map_stride == 0;
    if (shared_map && o.n_lines > 0) {
        rc = reserve_scratch(h, align_up(sizeof(uint32_t) * (size_t)o.n_lines) + kAlign);
        if (rc != WH_OK) return rc;
        a.line_key = static_cast<uint32_t*>(h->scratch);
        if (wh::launch_prep(a, s) != cudaSuccess) return WH_ECUDA;
    }
    wh::FeatConst c;
    c.A = h->g.A;
    c.L = h->g.L;
    c.magic_a = (((uint64_t)1 << 40) + (uint64_t)h->g.A - 1) / (uint64_t)h->g.A;
    c.magic_l = (((uint64_t)1 << 40) + (uint64_t)h->g.L - 1) / (uint64_t)h->g.L;
    c.inv_a = (float)(1.0 / (double)h->g.A);
    return wh::launch_features(a, c, X, nullptr, p.n_tours, h->num_sms, s) == cudaSuccess ? WH_OK : WH_ECUDA;
}

extern "C" int wh_batch_grow(wh_layout* h, const wh_orders* orders, const int32_t* slot_map,
                             int64_t slot_map_stride, int32_t n_maps, int32_t max_orders, int32_t max_lines,
                             int32_t* tour_off, int32_t* order_seq, int32_t* n_tours, void* stream) {
    if (!h || !orders || n_maps < 0 || max_orders < 0 || max_lines < 0 || slot_map_stride < 0) return WH_EINVAL;
    if (n_maps == 0) return WH_OK;
    const wh_orders o = *orders;
    if (!slot_map || !tour_off || !order_seq || !n_tours || !o.order_off || (o.n_lines > 0 && !o.line_sku) ||
        o.n_orders < 0 || o.n_lines < 0 || o.n_sku < 1)
        return WH_EINVAL;
    if (slot_map_stride != 0 && slot_map_stride < o.n_sku) return WH_EINVAL;
    if (h->g.A > 255 || h->g.L > 256) return WH_ERANGE;   // 16-bit keys, 256-bit depth masks
    if (o.n_orders > 65535) return WH_ERANGE;   // 16-bit order ids in the unassigned list
    if (wh::batch_grow_smem_bytes(o.n_orders, o.n_lines, h->g.A) > 200 * 1024) return WH_ERANGE;
    int rc = bind_device(h);
    if (rc != WH_OK) return rc;
    wh::BatchGrowArgs B;
    std::memset(&B, 0, sizeof(B));
    wh_plans p;
    std::memset(&p, 0, sizeof(p));
    p.slot_map = slot_map;
    p.slot_map_stride = slot_map_stride;
    wh_costs none;
    std::memset(&none, 0, sizeof(none));
    fill_args(B.a, h->g, o, p, none, WH_ROUTE_OPTIMAL);
    B.a.status = h->meta;
    B.max_orders = max_orders;
    B.max_lines = max_lines;
    B.tour_off = tour_off;
    B.order_seq = order_seq;
    B.n_tours = n_tours;
    return wh::launch_batch_grow(B, n_maps, static_cast<cudaStream_t>(stream)) == cudaSuccess ? WH_OK : WH_ECUDA;
}

extern "C" int wh_occupancy(wh_layout* h, const wh_orders* orders, const wh_plans* plans, void* stream) {
    if (!h || !orders || !plans) return WH_EINVAL;
    const wh_orders o = *orders;
    const wh_plans p = *plans;
    if (p.n_plans < 0 || o.n_sku < 0 || p.slot_map_stride < o.n_sku || p.slot_map_stride <= 0) return WH_EINVAL;
    if (p.n_plans == 0) return WH_OK;
    if (!p.loc_used || (o.n_sku > 0 && !p.slot_map)) return WH_EINVAL;
    int rc = bind_device(h);
    if (rc != WH_OK) return rc;
    return wh::launch_occupancy(p.slot_map, p.slot_map_stride, p.n_plans, o.n_sku, h->g.n_loc, p.loc_used,
                                h->num_sms, static_cast<cudaStream_t>(stream)) == cudaSuccess
               ? WH_OK
               : WH_ECUDA;
}

extern "C" int wh_kmeans_slotting(wh_layout* h, const wh_orders* orders, const int8_t* signs, int32_t freq_weight,
                                  int32_t k, const int32_t* init, const uint64_t* u, int32_t iters, int32_t* x_out,
                                  int32_t* init_out, int32_t* centroids, int32_t* assign, int32_t* slot_map,
                                  void* stream) {
    if (!h || !orders || !signs || !centroids || !assign || !slot_map || (!init && !u)) return WH_EINVAL;
    const wh_orders o = *orders;
    if (o.n_orders < 0 || o.n_lines < 0 || o.n_sku < 1 || !o.order_off || (o.n_lines > 0 && !o.line_sku))
        return WH_EINVAL;
    if (k < 1 || k > o.n_sku || iters < 0 || freq_weight < 0) return WH_EINVAL;
    if (k > wh::KM_MAX_K || freq_weight > wh::KM_MAX_FREQ_WEIGHT || o.n_lines >= (1 << 26)) return WH_ERANGE;
    if ((int64_t)o.n_sku > (int64_t)h->g.n_loc) return WH_ERANGE;
    if ((reinterpret_cast<uintptr_t>(signs) & 15) != 0 || (reinterpret_cast<uintptr_t>(x_out) & 15) != 0)
        return WH_EINVAL;
    int rc = bind_device(h);
    if (rc != WH_OK) return rc;
    const size_t n = (size_t)o.n_sku, K = (size_t)k;
    const size_t nb = (n + 255) / 256;
    const size_t sz[] = {
        align_up(8 * n * wh::KM_DIM),             // co
        align_up(4 * n),                          // freq
        x_out ? 0 : align_up(4 * n * wh::KM_DIM), // x
        init ? 0 : align_up(8 * n),               // dmin
        init ? 0 : align_up(8 * nb),              // bsum
        align_up(4),                              // done
        init_out ? 0 : align_up(4 * K),           // seeds
        align_up(8 * K * wh::KM_DIM),             // sum
        align_up(4 * K),                          // cnt
        align_up(8 * K),                          // weight
        align_up(4 * K),                          // off
        align_up(4 * K),                          // cur
        align_up(4 * (K + 1)),                    // off_by_rank
        align_up(8 * n),                          // mkey
    };
    size_t total = 0;
    for (size_t v : sz) total += v;
    rc = reserve_scratch(h, total);
    if (rc != WH_OK) return rc;
    char* q = static_cast<char*>(h->scratch);
    auto take = [&](size_t bytes) -> void* {
        void* r = bytes ? q : nullptr;
        q += bytes;
        return r;
    };
    wh::KmArgs A;
    std::memset(&A, 0, sizeof(A));
    A.g = h->g;
    A.n_orders = o.n_orders;
    A.n_lines = o.n_lines;
    A.n_sku = o.n_sku;
    A.order_off = o.order_off;
    A.line_sku = o.line_sku;
    A.signs = signs;
    A.fw = freq_weight;
    A.k = k;
    A.iters = iters;
    A.init = init;
    A.u = u;
    A.co = static_cast<long long*>(take(sz[0]));
    A.freq = static_cast<int32_t*>(take(sz[1]));
    A.x = x_out ? x_out : static_cast<int32_t*>(take(sz[2]));
    A.dmin = static_cast<long long*>(take(sz[3]));
    A.bsum = static_cast<long long*>(take(sz[4]));
    A.done = static_cast<unsigned int*>(take(sz[5]));
    A.seeds = init_out ? init_out : static_cast<int32_t*>(take(sz[6]));
    A.cent = centroids;
    A.sum = static_cast<long long*>(take(sz[7]));
    A.cnt = static_cast<int32_t*>(take(sz[8]));
    A.weight = static_cast<long long*>(take(sz[9]));
    A.off = static_cast<int32_t*>(take(sz[10]));
    A.cur = static_cast<int32_t*>(take(sz[11]));
    A.off_by_rank = static_cast<int32_t*>(take(sz[12]));
    A.mkey = static_cast<unsigned long long*>(take(sz[13]));
    A.assign = assign;
    A.slot_map = slot_map;
    A.status = h->meta;
    return wh::launch_kmeans(A, static_cast<cudaStream_t>(stream)) == cudaSuccess ? WH_OK : WH_ECUDA;
}

extern "C" int wh_routes(wh_layout* h, const wh_orders* orders, const wh_plans* plans, const int32_t* tours,
                         int32_t n, int32_t max_points, int32_t* points, int32_t* n_points, int32_t* length,
                         void* stream) {
    if (!h || !orders || !plans || n < 0 || max_points < 0) return WH_EINVAL;
    const wh_orders o = *orders;
    const wh_plans p = *plans;
    int rc = check_problem(o, p);
    if (rc != WH_OK) return rc;
    if (n == 0) return WH_OK;
    if (!tours || !n_points || !length || (max_points > 0 && !points)) return WH_EINVAL;
    if (p.slot_map_stride != 0 && (p.n_plans < 1 || !p.plan_tour_off)) return WH_EINVAL;
    rc = bind_device(h);
    if (rc != WH_OK) return rc;
    wh::EvalArgs a;
    wh_costs none;
    std::memset(&none, 0, sizeof(none));
    fill_args(a, h->g, o, p, none, WH_ROUTE_OPTIMAL);
    a.status = h->meta;
    return wh::launch_routes(a, tours, n, max_points, points, n_points, length, static_cast<cudaStream_t>(stream)) ==
                   cudaSuccess
               ? WH_OK
               : WH_ECUDA;
}

extern "C" int wh_widen_u16(const uint16_t* src, int32_t* dst, int64_t n, void* stream) {
    if (n < 0 || (n > 0 && (!src || !dst))) return WH_EINVAL;
    return wh::launch_widen_u16(src, dst, n, static_cast<cudaStream_t>(stream)) == cudaSuccess ? WH_OK : WH_ECUDA;
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

extern "C" int wh_get_move_stats(wh_layout* h, void* stream, int64_t* tours, int64_t* lines) {
    if (!h || !tours || !lines) return WH_EINVAL;
    if (!h->meta) {
        *tours = *lines = 0;
        return WH_OK;
    }
    DeviceGuard guard(h->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned long long v[2] = {0, 0};
    if (cudaMemcpyAsync(v, h->meta + 4, sizeof(v), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return WH_ECUDA;
    *tours = (int64_t)v[0];
    *lines = (int64_t)v[1];
    return WH_OK;
}

extern "C" int wh_set_timing(wh_layout* h, int enable) {
    if (!h) return WH_EINVAL;
    h->timing.on = enable != 0;
    h->timing.n = 0;
    return WH_OK;
}

extern "C" int wh_get_timing(wh_layout* h, int32_t* n_kernels, const char** names, int32_t* launches,
                             double* total_ms, int32_t cap) {
    if (!h || !n_kernels || cap < 0 || (cap > 0 && (!names || !launches || !total_ms))) return WH_EINVAL;
    DeviceGuard guard(h->device);
    return read_timing(h->timing, K_COUNT, kKernelNames, n_kernels, names, launches, total_ms, cap);
}

extern "C" void wh_destroy(wh_layout* h) {
    if (!h) return;
    if (h->device >= 0) {
        DeviceGuard guard(h->device);
        free_timing(h->timing);
        if (h->mv_scratch) cudaFree(h->mv_scratch);
        if (h->mv_tasks) cudaFree(h->mv_tasks);
        if (h->mv_long) cudaFree(h->mv_long);
        if (h->sr_scratch) cudaFree(h->sr_scratch);
        if (h->scratch) cudaFree(h->scratch);
        if (h->meta) cudaFree(h->meta);
    }
    delete h;
}

// ---------------------------------------------------------------- batches

namespace {

void drop_graphs(wh_batch* b) {
    for (auto& g : b->graphs) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
}

// Work items: each instance's 32-tour chunks cut into runs of
// chunks_per_item, ordered by estimated cost (chunks x orders per tour),
// largest first; ties keep instance order, so the order is deterministic.
int build_items(wh_batch* b) {
    std::vector<wh::WorkItem> items;
    for (int32_t i = 0; i < b->n_inst; ++i) {
        const wh::EvalArgs& a = b->args[i];
        const int32_t chunks = (a.n_tours + 31) / 32;
        const int64_t per_chunk = a.n_tours > 0 ? std::max<int64_t>(1, a.n_seq / std::max(1, a.n_tours)) : 1;
        for (int32_t c = 0; c < chunks; c += b->chunks_per_item) {
            wh::WorkItem w;
            w.inst = i;
            w.chunk_begin = c;
            w.chunk_end = std::min(chunks, c + b->chunks_per_item);
            w.cost = (int32_t)std::min<int64_t>(0x7fffffff, (int64_t)(w.chunk_end - w.chunk_begin) * per_chunk);
            items.push_back(w);
        }
    }
    std::stable_sort(items.begin(), items.end(),
                     [](const wh::WorkItem& x, const wh::WorkItem& y) { return x.cost > y.cost; });
    if (items.size() > b->items_cap) {
        if (b->d_items) cudaFree(b->d_items);
        b->d_items = nullptr;
        b->items_cap = 0;
        if (cudaMalloc(&b->d_items, sizeof(wh::WorkItem) * std::max<size_t>(items.size(), 1)) != cudaSuccess) {
            cudaGetLastError();
            return WH_ENOMEM;
        }
        b->items_cap = items.size();
    }
    if (!items.empty() &&
        cudaMemcpy(b->d_items, items.data(), sizeof(wh::WorkItem) * items.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return WH_ECUDA;
    b->n_items = (int32_t)items.size();
    drop_graphs(b);
    return WH_OK;
}

wh::BatchArgs batch_args(const wh_batch* b, uint32_t mask) {
    wh::BatchArgs B;
    B.insts = b->d_args;
    B.n_inst = b->n_inst;
    B.items = b->d_items;
    B.n_items = b->n_items;
    B.queue = reinterpret_cast<int32_t*>(b->meta + 2);
    B.long_count = reinterpret_cast<int32_t*>(b->meta + 1);
    B.mask = mask;
    B.max_orders = b->max_orders;
    B.max_lines = b->max_lines;
    B.max_rec = b->max_rec;
    B.id16 = b->id16 ? 1 : 0;
    return B;
}

enum BatchKernelId { KB_PREP = 0, KB_EVAL = 1, KB_LONG = 2, KB_COUNT = 3 };
const char* const kBatchKernelNames[KB_COUNT] = {"k_prep_batch", "k_eval_batch", "k_eval_long"};

// The batch's launch sequence; `timed`: bracket each launch with the batch's
// timing events when its timing is on (never while capturing a graph)
int launch_batch(wh_batch* b, uint32_t mask, cudaStream_t s, bool timed = false) {
    KernelTiming off;
    KernelTiming& tm = timed ? b->timing : off;
    const wh::BatchArgs B = batch_args(b, mask);
    {
        LaunchTimer lt(tm, KB_PREP, s);
        if (wh::launch_prep_batch(B, b->max_work, s) != cudaSuccess) return WH_ECUDA;
    }
    {
        LaunchTimer lt(tm, KB_EVAL, s);
        if (wh::launch_eval_batch(B, b->tune, b->key16, b->num_sms, s) != cudaSuccess) return WH_ECUDA;
    }
    wh::LongArgs L;
    std::memset(&L, 0, sizeof(L));
    L.insts = b->d_args;
    L.list = b->args.empty() ? nullptr : b->args[0].long_list;
    L.count = B.long_count;
    L.cap = b->long_cap;
    L.mask = mask;
    L.rec = b->long_rec;
    LaunchTimer lt(tm, KB_LONG, s);
    if (wh::launch_eval_long(L, true, b->num_sms, s) != cudaSuccess) return WH_ECUDA;
    return WH_OK;
}

bool valid_mask(uint32_t m) { return m != 0 && !(m & ~(WH_ROUTE_SSHAPE | WH_ROUTE_OPTIMAL)); }

}  // namespace

extern "C" int wh_batch_create(const wh_instance* insts, int32_t n, wh_batch** out) {
    if (!insts || n < 1 || !out) return WH_EINVAL;
    wh_batch* b = new (std::nothrow) wh_batch;
    if (!b) return WH_ENOMEM;
    int rc = device_info(&b->device, &b->num_sms);
    if (rc != WH_OK) {
        b->device = -1;
        delete b;
        return rc;
    }
    b->n_inst = n;
    b->args.resize(n);
    size_t key_bytes = 0;
    // 16-bit order ids: every instance or none (one kernel reads them all)
    int n16 = 0;
    for (int32_t i = 0; i < n; ++i) n16 += insts[i].order_seq16 != nullptr;
    b->id16 = n16 == n;
    for (int32_t i = 0; i < n; ++i) {
        wh::Geo g;
        rc = check_desc(insts[i].layout, &g);
        wh_plans p = insts[i].plans;
        if (b->id16) {
            if (insts[i].orders.n_orders > 65536) rc = WH_EINVAL;
            p.order_seq = reinterpret_cast<const int32_t*>(insts[i].order_seq16);   // presence check only
        }
        if (n16 != 0 && n16 != n) rc = WH_EINVAL;
        if (rc == WH_OK) rc = check_problem(insts[i].orders, p);
        if (rc == WH_OK && (p.slot_map_stride != 0 || p.n_plans < 1)) rc = WH_EINVAL;
        if (rc != WH_OK) {
            b->device = -1;
            delete b;
            return rc;
        }
        fill_args(b->args[i], g, insts[i].orders, insts[i].plans, insts[i].out, WH_ROUTE_SSHAPE | WH_ROUTE_OPTIMAL);
        if (b->id16) {
            b->args[i].order_seq = nullptr;
            b->args[i].order_seq16 = insts[i].order_seq16;
        }
        b->key16 = b->key16 && wh::key16_ok(g);
        b->max_orders = std::max(b->max_orders, insts[i].orders.n_orders);
        b->max_lines = std::max(b->max_lines, insts[i].orders.n_lines);
        b->max_rec = std::max(b->max_rec, b->args[i].max_rec);
        b->max_work = std::max(b->max_work, std::max(insts[i].orders.n_lines, insts[i].plans.n_plans));
        b->total_tours += insts[i].plans.n_tours;
        key_bytes += align_up(sizeof(uint32_t) * (size_t)insts[i].orders.n_lines);
    }
    b->long_cap = (int32_t)std::min<int64_t>(kBatchLongCap, b->total_tours + 1);
    const size_t list_bytes = align_up(sizeof(int32_t) * 3 * (size_t)b->long_cap);
    const size_t rec_bytes = align_up(wh::long_rec_bytes(b->num_sms));
    if (cudaMalloc(&b->meta, kAlign) != cudaSuccess || cudaMemset(b->meta, 0, kAlign) != cudaSuccess ||
        cudaMalloc(&b->scratch, key_bytes + list_bytes + rec_bytes) != cudaSuccess ||
        cudaMalloc(&b->d_args, sizeof(wh::EvalArgs) * n) != cudaSuccess) {
        cudaGetLastError();
        wh_batch_destroy(b);
        return WH_ENOMEM;
    }
    char* base = static_cast<char*>(b->scratch);
    int32_t* list = reinterpret_cast<int32_t*>(base + key_bytes);
    b->long_rec = rec_bytes ? reinterpret_cast<uint2*>(base + key_bytes + list_bytes) : nullptr;
    size_t off = 0;
    for (int32_t i = 0; i < n; ++i) {
        wh::EvalArgs& a = b->args[i];
        a.line_key = a.n_lines > 0 ? reinterpret_cast<uint32_t*>(base + off) : nullptr;
        off += align_up(sizeof(uint32_t) * (size_t)a.n_lines);
        a.status = b->meta;
        a.long_count = reinterpret_cast<int32_t*>(b->meta + 1);
        a.long_list = list;
        a.long_cap = b->long_cap;
    }
    if (cudaMemcpy(b->d_args, b->args.data(), sizeof(wh::EvalArgs) * n, cudaMemcpyHostToDevice) != cudaSuccess) {
        wh_batch_destroy(b);
        return WH_ECUDA;
    }
    b->tune.threads = 256;
    b->tune.key16 = b->key16 ? 1 : 0;
    b->tune.smem_tables = 1;
    if (wh::eval_batch_smem_bytes(batch_args(b, 3), b->tune, b->key16) > 112 * 1024) b->tune.smem_tables = 0;
    b->chunks_per_item = 16;
    rc = build_items(b);
    if (rc != WH_OK) {
        wh_batch_destroy(b);
        return rc;
    }
    *out = b;
    return WH_OK;
}

extern "C" int wh_batch_set_tuning(wh_batch* b, int32_t threads, int32_t chunks_per_item, int32_t smem_tables) {
    if (!b || threads < 32 || threads > (b->key16 ? 384 : 256) || (threads % 32) || chunks_per_item < 1 ||
        smem_tables < 0 ||
        smem_tables > 1)
        return WH_EINVAL;
    DeviceGuard guard(b->device);
    wh::Tuning t = b->tune;
    t.threads = threads;
    t.smem_tables = smem_tables;
    if (t.smem_tables && wh::eval_batch_smem_bytes(batch_args(b, 3), t, b->key16) > 200 * 1024) t.smem_tables = 0;
    b->tune = t;
    if (chunks_per_item != b->chunks_per_item) {
        b->chunks_per_item = chunks_per_item;
        return build_items(b);
    }
    drop_graphs(b);
    return WH_OK;
}

extern "C" int wh_batch_get_tuning(wh_batch* b, int32_t* threads, int32_t* chunks_per_item, int32_t* smem_tables) {
    if (!b || !threads || !chunks_per_item || !smem_tables) return WH_EINVAL;
    *threads = b->tune.threads;
    *chunks_per_item = b->chunks_per_item;
    *smem_tables = b->tune.smem_tables;
    return WH_OK;
}

extern "C" int wh_batch_eval(wh_batch* b, uint32_t routing_mask, void* stream) {
    if (!b || !valid_mask(routing_mask)) return WH_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return WH_ECUDA;
    if (dev != b->device) return WH_EINVAL;
    return launch_batch(b, routing_mask, static_cast<cudaStream_t>(stream), true);
}

extern "C" int wh_batch_set_timing(wh_batch* b, int enable) {
    if (!b) return WH_EINVAL;
    b->timing.on = enable != 0;
    b->timing.n = 0;
    return WH_OK;
}

extern "C" int wh_batch_get_timing(wh_batch* b, int32_t* n_kernels, const char** names, int32_t* launches,
                                   double* total_ms, int32_t cap) {
    if (!b || !n_kernels || cap < 0 || (cap > 0 && (!names || !launches || !total_ms))) return WH_EINVAL;
    DeviceGuard guard(b->device);
    return read_timing(b->timing, KB_COUNT, kBatchKernelNames, n_kernels, names, launches, total_ms, cap);
}

extern "C" int wh_batch_eval_graph(wh_batch* b, uint32_t routing_mask, void* stream) {
    if (!b || !valid_mask(routing_mask)) return WH_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return WH_ECUDA;
    if (dev != b->device) return WH_EINVAL;
    cudaGraphExec_t& exec = b->graphs[routing_mask];
    if (!exec) {
        if (!b->capture && cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking) != cudaSuccess) return WH_ECUDA;
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return WH_ECUDA;
        const int rc = launch_batch(b, routing_mask, b->capture);
        const cudaError_t ec = cudaStreamEndCapture(b->capture, &graph);
        if (rc != WH_OK || ec != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return rc != WH_OK ? rc : WH_ECUDA;
        }
        const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            exec = nullptr;
            return WH_ECUDA;
        }
    }
    return cudaGraphLaunch(exec, static_cast<cudaStream_t>(stream)) == cudaSuccess ? WH_OK : WH_ECUDA;
}

namespace {

// The autotune cache is a flat JSON object, one entry per size bucket:
//   {"<bucket>": {"threads": T, "chunks_per_item": C, "ms": X}, ...}
struct TuneEntry {
    int threads = 0, chunks = 0;
    double ms = 0;
};

std::map<std::string, TuneEntry> read_cache(const char* path) {
    std::map<std::string, TuneEntry> m;
    FILE* f = path ? std::fopen(path, "r") : nullptr;
    if (!f) return m;
    std::string text;
    char buf[4096];
    size_t k;
    while ((k = std::fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, k);
    std::fclose(f);
    size_t pos = 0;
    while ((pos = text.find('"', pos)) != std::string::npos) {
        const size_t end = text.find('"', pos + 1);
        if (end == std::string::npos) break;
        const std::string key = text.substr(pos + 1, end - pos - 1);
        const size_t brace = text.find('{', end);
        const size_t close = text.find('}', end);
        if (brace == std::string::npos || close == std::string::npos || brace > close) {
            pos = end + 1;
            continue;
        }
        const std::string body = text.substr(brace, close - brace + 1);
        TuneEntry e;
        const size_t ti = body.find("\"threads\"");
        const size_t ci = body.find("\"chunks_per_item\"");
        const size_t mi = body.find("\"ms\"");
        if (ti != std::string::npos && ci != std::string::npos) {
            e.threads = std::atoi(body.c_str() + body.find(':', ti) + 1);
            e.chunks = std::atoi(body.c_str() + body.find(':', ci) + 1);
            if (mi != std::string::npos) e.ms = std::atof(body.c_str() + body.find(':', mi) + 1);
            m[key] = e;
        }
        pos = close + 1;
    }
    return m;
}

bool write_cache(const char* path, const std::map<std::string, TuneEntry>& m) {
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "w");
    if (!f) return false;
    std::fprintf(f, "{\n");
    size_t i = 0;
    for (const auto& kv : m) {
        std::fprintf(f, "  \"%s\": {\"threads\": %d, \"chunks_per_item\": %d, \"ms\": %.6f}%s\n", kv.first.c_str(),
                     kv.second.threads, kv.second.chunks, kv.second.ms, ++i < m.size() ? "," : "");
    }
    std::fprintf(f, "}\n");
    std::fclose(f);
    return std::rename(tmp.c_str(), path) == 0;
}

int ilog2(int64_t v) {
    int r = 0;
    while (v > 1) {
        v >>= 1;
        ++r;
    }
    return r;
}

std::string bucket_key(const wh_batch* b, uint32_t mask) {
    char k[160];
    std::snprintf(k, sizeof(k), "key%d_inst2^%d_tours2^%d_orders2^%d_mask%u", b->key16 ? 16 : 32, ilog2(b->n_inst),
                  ilog2(std::max<int64_t>(1, b->total_tours)), ilog2(std::max(1, b->max_orders)), mask);
    return k;
}

}  // namespace

extern "C" int wh_batch_autotune(wh_batch* b, uint32_t routing_mask, const char* cache_path, void* stream,
                                 int32_t* threads, int32_t* chunks_per_item, int32_t* from_cache) {
    if (!b || !valid_mask(routing_mask)) return WH_EINVAL;
    DeviceGuard guard(b->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const std::string key = bucket_key(b, routing_mask);
    std::map<std::string, TuneEntry> cache = read_cache(cache_path);
    auto it = cache.find(key);
    int rc = WH_OK;
    if (it != cache.end() && it->second.threads > 0 && it->second.chunks > 0) {
        rc = wh_batch_set_tuning(b, it->second.threads, it->second.chunks, b->tune.smem_tables);
        if (from_cache) *from_cache = 1;
    } else {
        if (from_cache) *from_cache = 0;
        const int32_t smem = b->tune.smem_tables;
        const int thread_opts[] = {128, 256, 384};
        // powers of two, and for a warp count that is not one (384 threads:
        // 12 warps) the multiples of the warp count that split an item's
        // chunks evenly over the CTA's warps
        const int chunk_opts[] = {2, 4, 8, 16, 32, 64, 128, 256, 512, 1024, 2048, 4096};
        const int warp_mults[] = {1, 2, 4, 8, 16, 32, 64, 128};
        cudaEvent_t e0, e1;
        if (cudaEventCreate(&e0) != cudaSuccess) return WH_ECUDA;
        if (cudaEventCreate(&e1) != cudaSuccess) {
            cudaEventDestroy(e0);
            return WH_ECUDA;
        }
        TuneEntry best;
        best.ms = 1e30;
        for (int th : thread_opts) {
            if (th > 256 && !b->key16) continue;
            std::vector<int> chs(std::begin(chunk_opts), std::end(chunk_opts));
            const int nw = th / 32;
            if (nw & (nw - 1))
                for (int m : warp_mults) chs.push_back(nw * m);
            for (int ch : chs) {
                rc = wh_batch_set_tuning(b, th, ch, smem);
                if (rc != WH_OK) break;
                rc = launch_batch(b, routing_mask, s);   // warm-up
                if (rc != WH_OK) break;
                cudaEventRecord(e0, s);
                for (int r = 0; r < 3 && rc == WH_OK; ++r) rc = launch_batch(b, routing_mask, s);
                cudaEventRecord(e1, s);
                if (rc != WH_OK || cudaEventSynchronize(e1) != cudaSuccess) {
                    rc = rc != WH_OK ? rc : WH_ECUDA;
                    break;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms / 3 < best.ms) {
                    best.ms = ms / 3;
                    best.threads = th;
                    best.chunks = ch;
                }
            }
            if (rc != WH_OK) break;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rc != WH_OK) return rc;
        rc = wh_batch_set_tuning(b, best.threads, best.chunks, smem);
        if (rc == WH_OK && cache_path) {
            cache[key] = best;
            write_cache(cache_path, cache);
        }
    }
    if (threads) *threads = b->tune.threads;
    if (chunks_per_item) *chunks_per_item = b->chunks_per_item;
    return rc;
}

extern "C" int wh_batch_get_status(wh_batch* b, void* stream, uint32_t* status) {
    if (!b || !status) return WH_EINVAL;
    DeviceGuard guard(b->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t v = 0;
    if (cudaMemcpyAsync(&v, b->meta, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess) return WH_ECUDA;
    if (cudaMemsetAsync(b->meta, 0, sizeof(uint32_t), s) != cudaSuccess) return WH_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return WH_ECUDA;
    *status = v;
    return WH_OK;
}

extern "C" void wh_batch_destroy(wh_batch* b) {
    if (!b) return;
    if (b->device >= 0) {
        DeviceGuard guard(b->device);
        drop_graphs(b);
        free_timing(b->timing);
        if (b->capture) cudaStreamDestroy(b->capture);
        if (b->d_items) cudaFree(b->d_items);
        if (b->d_args) cudaFree(b->d_args);
        if (b->scratch) cudaFree(b->scratch);
        if (b->meta) cudaFree(b->meta);
    }
    delete b;
}
