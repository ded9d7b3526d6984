// Internal declarations shared by the C-ABI host code and the kernels.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/wh.h"

namespace wh {

// packed pick key: aisle in the high 16 bits, slot index k in the low 16;
// ascending key order = ascending (aisle, depth)
constexpr uint32_t KEY_NONE = 0xFFFFFFFFu;
constexpr int SHORT_MAX = 64;   // tours up to this many lines run one per thread

struct Geo {
    int32_t A, L, P, S, W;
    int32_t h;      // W/2: depth of slot 0
    int32_t Y;      // back cross-aisle depth
    int32_t n_loc;  // A*2*L
    // exact division of a location (0 <= loc < 2^31) by 2L:
    // loc / 2L = umulhi(loc, div_m) >> div_s (Granlund & Montgomery,
    // "Division by invariant integers using multiplication", 1994: with
    // l = ceil(log2 2L) and div_m = ceil(2^(31+l) / 2L) < 2^32 the quotient is
    // exact for every numerator below 2^31); set by geo_set_div
    uint32_t div_m;
    int32_t div_s;
};

inline void geo_set_div(Geo& g) {
    const uint64_t d = 2ull * (uint64_t)g.L;
    int l = 0;
    while ((1ull << l) < d) ++l;   // ceil(log2 d); d >= 2
    g.div_m = (uint32_t)(((1ull << (31 + l)) + d - 1) / d);
    g.div_s = l - 1;
}

struct EvalArgs {
    Geo g;
    int32_t n_orders, n_lines, n_sku;
    const int32_t* order_off;
    const int32_t* line_sku;
    const uint32_t* line_key;   // shared slotting: key of every line (scratch)
    const int32_t* slot_map;
    int64_t slot_stride;        // 0: shared slotting
    uint32_t* loc_used;         // per-plan occupancy bits or null (relocation moves)
    int32_t n_plans, n_tours;
    int64_t n_seq;
    const int32_t* plan_tour_off;
    const int32_t* tour_off;
    const int32_t* order_seq;
    const uint16_t* order_seq16;   // the order ids as 16-bit values (batched instances), else NULL
    int32_t* tour_s;
    int32_t* tour_rr;
    int64_t* plan_s;
    int64_t* plan_rr;
    uint32_t mask;
    int32_t max_rec;            // record slots per thread (a tour with more pick aisles goes to the long pass)
    uint32_t* status;           // device status word
    int32_t* long_list;         // tours deferred to the long-tour kernel: (inst, tour, plan)
    int32_t* long_count;
    int32_t long_cap;           // capacity of long_list in entries
    // S-shape only under a shared slotting on at most 64 aisles: per order
    // {visited-aisle bits 0-31, bits 32-63, largest key, flags} built by
    // k_prep (flags: 1 invalid line, 2 has lines, 4 invalid offsets); NULL
    // otherwise
    uint4* order_agg;
};

// A work item of the batched launch: 32-tour chunks [chunk_begin, chunk_end)
// of instance `inst`.
struct WorkItem {
    int32_t inst;
    int32_t chunk_begin;
    int32_t chunk_end;
    int32_t cost;               // estimated work, for the largest-first order
};

struct BatchArgs {
    const EvalArgs* insts;      // device array, one per instance
    int32_t n_inst;
    const WorkItem* items;      // device array, largest first
    int32_t n_items;
    int32_t* queue;             // next item to take (zeroed by the batch prep kernel)
    int32_t* long_count;
    uint32_t mask;
    int32_t max_orders, max_lines, max_rec;
    int32_t id16;               // every instance's order ids are 16-bit (order_seq16)
};

struct LongArgs {
    EvalArgs single;            // the instance when insts is NULL
    const EvalArgs* insts;      // batched instances (device), else NULL
    const int32_t* list;
    const int32_t* count;
    int32_t cap;
    uint32_t mask;
    // per-warp record scratch (long_rec_bytes): records are extracted in
    // parallel and the DPs of 32 tours run one per lane; NULL: each tour's
    // scan and DP run on one lane
    uint2* rec = nullptr;
};
// bytes of LongArgs::rec for a launch on num_sms SMs
size_t long_rec_bytes(int num_sms);

// Move evaluation (k_moves.cu)
struct MoveArgs {
    EvalArgs a;                 // the plans the moves apply to
    const int32_t* tour_s_old;  // current per-tour costs of those plans
    const int32_t* tour_rr_old;
    const int4* moves;          // {type, a, b, plan}
    int32_t n_moves;
    int32_t max_orders, max_lines;
    int64_t* delta;             // [n_moves][2]
    int32_t* mstatus;           // [n_moves]
    // scratch
    int32_t* order_tour;        // [n_plans][n_orders]: global tour holding the order, -1 if none
    int32_t* tour_lines;        // [n_tours]: lines of the tour, -1 if malformed
    int32_t* sku_off;           // [n_sku+1]: SKU -> orders index
    int32_t* sku_cur;           // [n_sku+1]: counts, then fill cursors
    int32_t* sku_orders;        // [n_lines]
    int64_t* task_off;          // [n_moves+1]: exclusive scan of task counts
    int64_t* scan_aux;          // block totals of that scan
    int4* tasks;                // [n_tasks]
    int2* task_cost;            // [n_tasks]: new (S-shape, optimal) cost of the task's tour, -1 if not counted
    int64_t n_tasks;
    int32_t* long_list;         // tasks over SHORT_MAX lines
    int32_t* long_count;
    int32_t long_cap;
    // long tasks' per-aisle records for the one-task-per-thread DP: record r
    // of list entry w at long_rec[r * long_rec_cap + w]; long_m[w] records
    // (-1: scored already), long_key[w] the largest key
    uint2* long_rec;
    int32_t* long_m;
    uint32_t* long_key;
    int32_t long_rec_cap;
    unsigned long long* stats;  // [0] changed tours walked, [1] their lines (zeroed by the count pass)
};

struct LsArgs {
    EvalArgs a;                 // plans edited in place (order_seq, tour_off, slot_map)
    const int4* moves;          // plan p owns moves [p*moves_per_plan, (p+1)*moves_per_plan)
    int32_t moves_per_plan;
    const int64_t* delta;
    const int32_t* status;
    int32_t* applied;           // [n_plans]
    int32_t seg_cap;            // shared-memory staging capacity (orders)
    // incremental cost update (all NULL: none): the tasks of the wh_eval_moves
    // call that scored these moves
    const int64_t* task_off;
    const int4* tasks;
    const int2* task_cost;
    int32_t* tour_s;
    int32_t* tour_rr;
    int64_t* plan_s;
    int64_t* plan_rr;
    uint8_t* tour_changed;      // NULL or set to 1 for every rewritten tour
};

struct ScreenArgs {
    MoveArgs M;                 // the scored moves and their task list
    const float* y_tour;        // predicted cost of every current tour
    const float* y_task;        // predicted cost of every task's changed tour
    float* score;               // [n_moves] predicted delta
    int32_t moves_per_plan;
    int32_t keep;
    int4* kept;                 // [n_plans][keep]
};

// seed-and-grow batch formation (k_batch.cu): one CTA per slotting
// a.slot_map + p * a.slot_stride; per slotting p, tour_off[p][n_orders + 1],
// order_seq[p][n_orders], n_tours[p]
struct BatchGrowArgs {
    EvalArgs a;
    int32_t max_orders, max_lines;
    int32_t* tour_off;
    int32_t* order_seq;
    int32_t* n_tours;
};
size_t batch_grow_smem_bytes(int n_orders, int n_lines, int A);
cudaError_t launch_batch_grow(const BatchGrowArgs& B, int n_maps, cudaStream_t s);

cudaError_t launch_occupancy(const int32_t* slot_map, int64_t stride, int32_t n_plans, int32_t n_sku, int32_t n_loc,
                             uint32_t* used, int num_sms, cudaStream_t st);

cudaError_t launch_widen_u16(const uint16_t* src, int32_t* dst, int64_t n, cudaStream_t s);

// K-means slotting (k_kmeans.cu)
constexpr int KM_DIM = 32;       // feature row: 31 sketch coordinates + the pick-count coordinate
constexpr int KM_SKETCH = 31;
constexpr int KM_SCALE = 1024;
constexpr int KM_MAX_K = 256;
constexpr int KM_MAX_FREQ_WEIGHT = 256;
struct KmArgs {
    Geo g;
    int32_t n_orders, n_lines, n_sku;
    const int32_t* order_off;
    const int32_t* line_sku;
    const int8_t* signs;         // [n_sku][32], column 31 unused
    int32_t fw, k, iters;
    const int32_t* init;         // [k] or null: K-means++ from u
    const uint64_t* u;           // [k]
    long long* co;               // [n_sku][32] scratch
    int32_t* freq;               // [n_sku]
    int32_t* x;                  // [n_sku][32]
    long long* dmin;             // [n_sku]
    long long* bsum;             // [blocks]
    unsigned int* done;
    int32_t* seeds;              // [k]
    int32_t* cent;               // [k][32]
    long long* sum;              // [k][32]
    int32_t* cnt;                // [k]
    long long* weight;           // [k]
    int32_t* off;                // [k]
    int32_t* cur;                // [k]
    int32_t* off_by_rank;        // [k + 1]
    unsigned long long* mkey;    // [n_sku]
    int32_t* assign;             // [n_sku]
    int32_t* slot_map;           // [n_sku]
    uint32_t* status;
};
size_t kmeans_assign_smem(int k);
cudaError_t launch_kmeans(const KmArgs& A, cudaStream_t s);

// explicit optimal routes of listed tours (k_route.cu)
constexpr int ROUTE_MAX_POINTS = 256;
cudaError_t launch_routes(const EvalArgs& a, const int32_t* tours, int32_t n, int32_t max_points, int32_t* points,
                          int32_t* n_points, int32_t* length, cudaStream_t s);

struct FeatConst;
cudaError_t launch_task_features(const MoveArgs& M, const FeatConst& c, void* X, int num_sms, cudaStream_t s);
cudaError_t launch_screen_select(const ScreenArgs& S, cudaStream_t s);

cudaError_t launch_ls_apply(const LsArgs& L, cudaStream_t s);
// the moves' index (order -> tour per plan, tour line counts, SKU -> orders),
// checks, task counts and offsets; reuse_index: the index of the same plans
// and order book is already in M's buffers, only the rest runs
cudaError_t launch_moves_prepare(const MoveArgs& M, int num_sms, cudaStream_t s, bool reuse_index);
// task fill + tasks of <= SHORT_MAX lines; the long ones are listed
cudaError_t launch_moves_eval(const MoveArgs& M, bool k16, int num_sms, cudaStream_t s);
// the listed long tasks (records, then their DPs) and the final status pass
cudaError_t launch_moves_long(const MoveArgs& M, int num_sms, cudaStream_t s);
constexpr int MVL_RMAX = 48;    // records per long task kept for the per-thread DP
cudaError_t launch_moves_fill(const MoveArgs& M, cudaStream_t s);

// Surrogate (k_surrogate.cu).  Packed parameter vector: w1 [192][256],
// b1 [256], w2 [256][256], b2 [256], w3 [256], b3 [1].
constexpr int64_t MLP_IN = 192;
constexpr int64_t MLP_W1 = 192 * 256;
constexpr int64_t MLP_B1_OFF = MLP_W1;
constexpr int64_t MLP_W2_OFF = MLP_B1_OFF + 256;
constexpr int64_t MLP_W2 = 256 * 256;
constexpr int64_t MLP_B2_OFF = MLP_W2_OFF + MLP_W2;
constexpr int64_t MLP_W3_OFF = MLP_B2_OFF + 256;
constexpr int64_t MLP_B3_OFF = MLP_W3_OFF + 256;
constexpr int64_t MLP_NPARAM = MLP_B3_OFF + 1;

// Training backward on the tensor cores (k_mlp_bwd.cu).  Row-major [n][256]
// buffers unless noted; the transposed copies are [features][ldt] bf16 with
// ldt a multiple of 64 (columns n .. ldt-1 unused: the tensor maps end at n).
struct BwdArgs {
    int64_t n;                  // rows of the batch
    int64_t ldt;                // row stride (elements) of the transposed copies
    const float* y;             // [n] outputs of the training forward
    const float* t;             // [n] targets
    const float* Z1;
    const float* Z2;
    const __nv_bfloat16* H1;
    const __nv_bfloat16* H2;
    const __nv_bfloat16* X;     // [n][192]
    const float* P;             // fp32 master parameters
    float* dy;                  // [n] (y - t) / n
    __nv_bfloat16* dZ2;
    __nv_bfloat16* H1T;         // [256][ldt]
    __nv_bfloat16* dZ2T;        // [256][ldt]
    __nv_bfloat16* XT;          // [193][ldt]: X transposed, row 192 = 1
    __nv_bfloat16* dZ1;
    __nv_bfloat16* dZ1T;        // [256][ldt]
    float* part_t;              // per 32-row block: b2[256], w3[256], b3, loss partial sums
    float* part_w;              // [2][splits][256][256]: dW2 and [dW1; db1] partial products
    int32_t splits;             // batch ranges of the weight gradients
    int64_t split_rows;         // rows per range (a multiple of 64)
    int* status;                // WH_STATUS_* bits (bounded waits)
};
int bwd_tail_part_floats(int64_t n);
cudaError_t launch_bwd(const BwdArgs& b, const CUtensorMap& mdz2, const CUtensorMap& mw2, const CUtensorMap& mh1t,
                       const CUtensorMap& mdz2t, const CUtensorMap& mxt, const CUtensorMap& mdz1t, int num_sms,
                       cudaStream_t s);
cudaError_t launch_adam_parts(const BwdArgs& b, float* p, float* m, float* v, float* G, float lr, int step, void* w1b,
                              void* w2b, float* loss, cudaStream_t s);

struct FeatConst {
    int32_t A, L;
    uint64_t magic_a;   // ceil(2^40 / A)
    uint64_t magic_l;   // ceil(2^40 / L)
    float inv_a;        // (float)(1.0 / A)
};
// features of tours list[0..n_rows) (list NULL: tours 0..n_rows) into rows 0..n_rows of X
cudaError_t launch_features(const EvalArgs& a, const FeatConst& c, void* X, const int32_t* list, int64_t n_rows,
                            int num_sms, cudaStream_t s);
cudaError_t launch_compact_flags(const uint8_t* flag, int64_t n, int32_t* list, int32_t* count, cudaStream_t s);
cudaError_t launch_scatter_pred(const int32_t* list, const float* y, int64_t n, float* y_tour, uint8_t* flag,
                                cudaStream_t s);
cudaError_t launch_to_bf16(const float* p, int64_t n, void* out, cudaStream_t s);
// fused tcgen05 inference (k_mlp_tc.cu): W1t [256][192] and W2t [256][256]
// are the transposed bf16 weights the tensor maps mw1 / mw2 describe
cudaError_t launch_transpose_bf16(const float* p, int K, int N, void* out, cudaStream_t s);
// Z1 / H1 / Z2 / H2 (all or none): the training forward's saved pre-
// activations (fp32) and activations (bf16), [n][256].  skip_tile / wait_ns:
// the bounded waits' test hook (skip_tile < 0 in normal use).
cudaError_t launch_mlp_tc(const CUtensorMap& mx, const CUtensorMap& mw1, const CUtensorMap& mw2, const float* P,
                          int64_t n, float* y, int* status, int num_sms, cudaStream_t s, float* Z1 = nullptr,
                          void* H1 = nullptr, float* Z2 = nullptr, void* H2 = nullptr, int64_t skip_tile = -1,
                          unsigned long long wait_ns = 0);
size_t mlp_tc_smem_bytes();

struct Tuning {
    int threads;          // CTA size: 32 tours in flight per warp
    int smem_tables;      // stage the order book (offsets + line keys) in shared memory
    int key16;            // 16-bit keys, two per register, when the layout allows
};

// launch wrappers (k_eval.cu)
bool key16_ok(const Geo& g);   // A <= 255 and L <= 256
// line keys (shared slotting, when a.line_key is set), zeroed plan sums and
// long-tour counter, plan offset checks
cudaError_t launch_prep(const EvalArgs& a, cudaStream_t s);
cudaError_t launch_prep_batch(const BatchArgs& b, int max_work, cudaStream_t s);
// routing mask S-shape only on a layout of at most 2,048 aisles: the
// sort-free S-shape kernel scores the short-tour pass (and every tour)
bool sshape_kernel_applies(const EvalArgs& a);
cudaError_t launch_eval_short(const EvalArgs& a, const Tuning& t, int num_sms, cudaStream_t s,
                              int* grid_out);
cudaError_t launch_eval_batch(const BatchArgs& b, const Tuning& t, bool k16, int num_sms, cudaStream_t s);
cudaError_t launch_eval_long(const LongArgs& L, bool shared_map, int num_sms, cudaStream_t s);
size_t eval_short_smem_bytes(const EvalArgs& a, const Tuning& t);
size_t eval_batch_smem_bytes(const BatchArgs& b, const Tuning& t, bool k16);

}  // namespace wh
