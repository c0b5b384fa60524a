// Internal declarations of the B300 timing library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <utility>
#include <vector>

#include "tdp.h"

namespace tdp {

// ---------------------------------------------------------------- errors ---
void set_error(const char *fmt, ...);

#define TDP_CUDA(call)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            tdp::set_error("%s:%d: %s failed: %s", __FILE__, __LINE__, #call,            \
                           cudaGetErrorString(e_));                                      \
            return TDP_ERR_CUDA;                                                         \
        }                                                                                \
    } while (0)

#define TDP_LAUNCH_CHECK() TDP_CUDA(cudaGetLastError())

#define TDP_TRY(call)                                                                    \
    do {                                                                                 \
        tdp_status s_ = (call);                                                          \
        if (s_ != TDP_OK) return s_;                                                     \
    } while (0)

// ------------------------------------------------------------- constants ---
constexpr int kMaxK = 32;          // paths per endpoint (one warp holds the frontier)
constexpr int kMaxFanin = 32;      // inputs of a combinational cell
constexpr int kBigFanout = 32;     // nets with more sinks are handled by a whole block
constexpr int kPre = 4;            // inputs / sinks whose loads are issued together
constexpr int kRedChunk = 64;       // endpoints per partial of the WNS / TNS reduction
constexpr int kCompactItems = 8192; // flags per block of the stream compaction
constexpr uint8_t kPfSmall = 1, kPfLarge = 2;  // net holds a pair sink; fanout <= / > kBigFanout
constexpr double kQScale = 16777216.0;  // 2^24: fixed point of slack/WNS in the pair update
constexpr double kQClamp = 32768.0;     // |slack/WNS| is clamped here before conversion

enum PinKind : uint8_t { PK_COMB_IN = 0, PK_ENDPOINT = 1, PK_COMB_OUT = 2, PK_START = 3 };

// flags of a combinational cell's input: its net is driven by a
// combinational cell; that driver is one level below the cell (level 0:
// flip-flops and primary inputs)
constexpr uint8_t kInComb = 1, kInPrev = 2;
// flag on a combinational input in the backward sweep's sink slots: its cell
// is one level above the net's driver
constexpr int kKindPrev = 0x10, kKindMask = 0x0f;

// Kernels that can be timed with tdp_profile_kernel (names in tdp_build.cu).
// The level sweeps are replayed from CUDA graphs: fwd_sweep is one replay of
// the forward level kernels, bwd_sweep one of the backward level kernels and
// the WNS / TNS reduction.
enum KernelId {
    KID_NET_RC, KID_FWD_SWEEP, KID_BWD_SWEEP, KID_VIOL_SORT, KID_TOPK, KID_PAIR_WALK,
    KID_PAIR_FINISH, KID_PP_FWD, KID_PP_BWD_NET, KID_PP_BWD_CELL, KID_RT_EXPAND, KID_EP_WNS,
    KID_INC_MOVED, KID_FWD_INC, KID_NET_WEIGHTS, KID_PP_FWD_BWD, KID_COUNT
};
extern const char *const kKernelNames[KID_COUNT];

// ------------------------------------------------- arrival accumulators ---
// FP32 graphs accumulate arrival and required times as an unevaluated sum of
// two floats (hi + lo, |lo| <= ulp(hi)/2): the delays themselves are FP32,
// but the long chains of additions keep their rounding error in lo, so the
// error stays relative to the delays rather than growing with the depth.
struct __align__(8) fx2 {
    float hi, lo;
};

template <typename R>
struct Acc;

template <>
struct Acc<double> {
    using T = double;
    static __host__ __device__ __forceinline__ T make(double v) { return v; }
    static __device__ __forceinline__ T add(T a, double b) { return a + b; }
    static __device__ __forceinline__ double diff(T a, T b) { return a - b; }
    static __device__ __forceinline__ bool gt(T a, T b) { return a > b; }
    static __device__ __forceinline__ bool lt(T a, T b) { return a < b; }
    static __device__ __forceinline__ double val(T a) { return a; }
    static __device__ __forceinline__ T ninf() { return -__longlong_as_double(0x7ff0000000000000ll); }
    static __device__ __forceinline__ T pinf() { return __longlong_as_double(0x7ff0000000000000ll); }
};

__device__ __forceinline__ fx2 fx2_add(fx2 a, float b) {
    // two-sum of a.hi + b, then fold in a.lo and renormalise (fast two-sum)
    float s = a.hi + b;
    float bb = s - a.hi;
    float err = (a.hi - (s - bb)) + (b - bb);
    float lo = a.lo + err;
    float hi = s + lo;
    lo = lo - (hi - s);
    return fx2{hi, lo};
}

template <>
struct Acc<float> {
    using T = fx2;
    static __host__ __device__ __forceinline__ T make(float v) { return fx2{v, 0.0f}; }
    static __device__ __forceinline__ T add(T a, float b) { return fx2_add(a, b); }
    static __device__ __forceinline__ float diff(T a, T b) {
        return (a.hi - b.hi) + (a.lo - b.lo);
    }
    static __device__ __forceinline__ bool gt(T a, T b) {
        return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo);
    }
    static __device__ __forceinline__ bool lt(T a, T b) {
        return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
    }
    static __device__ __forceinline__ float val(T a) { return a.hi + a.lo; }
    static __device__ __forceinline__ T ninf() { return fx2{-__int_as_float(0x7f800000), 0.0f}; }
    static __device__ __forceinline__ T pinf() { return fx2{__int_as_float(0x7f800000), 0.0f}; }
};

// Read-only loads through the non-coherent path.  Used for arrays a kernel
// never writes during its lifetime (topology, delays, and timing values of
// other levels, which earlier launches wrote).
template <typename T>
__device__ __forceinline__ T ldg(const T *p) { return __ldg(p); }
__device__ __forceinline__ fx2 ldg(const fx2 *p) {
    float2 v = __ldg(reinterpret_cast<const float2 *>(p));
    return fx2{v.x, v.y};
}

// Programmatic dependent launch (launch_pdl): a kernel lets its successor
// launch as soon as it starts (pdl_trigger), and the successor waits in
// pdl_wait() until every earlier kernel of the stream has finished and its
// writes are visible.  The per-level kernels of a sweep read only static
// topology before the wait.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// The kernels after the forward sweep (endpoints, extraction, pair update,
// loss) run as a chain of programmatic dependent launches: each lets the next
// launch once all of its blocks have started and then waits, before its
// first memory access, for every earlier kernel of the stream to finish.  So
// a kernel's launch and block dispatch overlap the tail of the one before,
// and the order of memory accesses is that of plain stream order (no read or
// write moves ahead of the wait).  A kernel whose predecessor in the stream
// is not a kernel (a memset, an event wait) starts as in plain stream order,
// and in a launch without the attribute both calls are no-ops.
__device__ __forceinline__ void chain_enter() {
    pdl_trigger();
    pdl_wait();
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), int grid, int block, cudaStream_t st,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// One sidetrack entry of a node's list: the deviation cost delta >= 0 of
// entering a node through a non-worst input pin instead of its worst one.
template <typename R>
struct __align__(2 * sizeof(R)) BEnt {
    R delta;
    int32_t pin;
};

__device__ __forceinline__ BEnt<float> ldg(const BEnt<float> *p) {
    float2 v = __ldg(reinterpret_cast<const float2 *>(p));
    return BEnt<float>{v.x, __float_as_int(v.y)};
}
__device__ __forceinline__ BEnt<double> ldg(const BEnt<double> *p) {
    double2 v = __ldg(reinterpret_cast<const double2 *>(p));
    return BEnt<double>{v.x, (int32_t)(__double_as_longlong(v.y) & 0xffffffffll)};
}

// Loads from L2, bypassing the (non-coherent) L1: for values another block of
// the same launch wrote before a grid-wide barrier.
template <typename T>
__device__ __forceinline__ T ldcg(const T *p) { return __ldcg(p); }
__device__ __forceinline__ fx2 ldcg(const fx2 *p) {
    float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
    return fx2{v.x, v.y};
}
__device__ __forceinline__ BEnt<float> ldcg(const BEnt<float> *p) {
    float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
    return BEnt<float>{v.x, __float_as_int(v.y)};
}
__device__ __forceinline__ BEnt<double> ldcg(const BEnt<double> *p) {
    double2 v = __ldcg(reinterpret_cast<const double2 *>(p));
    return BEnt<double>{v.x, (int32_t)(__double_as_longlong(v.y) & 0xffffffffll)};
}

// Load of a value written during the sweep: by an earlier launch (COH false,
// read-only path) or by another block of this launch (COH true, L2).
template <bool COH, typename T>
__device__ __forceinline__ T ldd(const T *p) {
    if constexpr (COH) return ldcg(p);
    else return ldg(p);
}

// Grid-wide barrier of a cooperative launch (every block resident).  count
// starts at zero for the launch and only grows; barrier n of the launch
// waits until it reaches n * gridDim.x.  A wait gives up after timeout_ns
// (or 2^26 polls), records status = 1 and every block leaves the kernel at
// its next barrier; the host reads status and reports TDP_ERR_TIMEOUT.
struct GridSync {
    unsigned *count = nullptr;
    unsigned *status = nullptr;
    unsigned long long timeout_ns = 0;
};
constexpr unsigned long long kSyncTimeoutNs = 200000000ull;  // 0.2 s per wait

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// grid_wait returns false (in every thread of the block) when the wait gave up.
// The barrier in two halves: grid_arrive (every thread; this block's writes
// become visible before its arrival is counted) and grid_wait (every
// thread); work that needs no other block's results of this step can run in
// between.  One thread of the block arrives and polls: lane 0 of its last
// warp (blockDim.x a multiple of 32).  The sweeps give their work to the
// first warps, so this thread's poll loads do not queue behind the loads
// the working warps issue between arrival and wait (measured: the forward
// sweep at 1.2M cells took 0.469 ms polling from thread 0, 0.426 ms from
// the last warp).
__device__ __forceinline__ bool grid_thread() { return threadIdx.x == blockDim.x - 32u; }

__device__ __forceinline__ void grid_arrive(const GridSync &gs) {
    __syncthreads();
    if (grid_thread()) {
        // release at GPU scope: this block's writes (ordered before by the
        // block barrier) become visible before the arrival is counted
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(gs.count) : "memory");
    }
}

__device__ __forceinline__ bool grid_wait(const GridSync &gs, unsigned target) {
    __shared__ int ok;
    if (grid_thread()) {
        int good = 1;
        unsigned long long t0 = 0;
        for (unsigned it = 1; ld_acquire(gs.count) < target; ++it) {
            if ((it & 255u) == 0u) {
                if (ld_acquire(gs.status) != 0u || it >= (1u << 26)) {
                    good = 0;
                    break;
                }
                const unsigned long long now = global_ns();
                if (t0 == 0ull) t0 = now;
                else if (now - t0 > gs.timeout_ns) {
                    atomicExch(gs.status, 1u);
                    good = 0;
                    break;
                }
            }
        }
        if (!good) atomicExch(gs.status, 1u);
        // no fence here: the acquire load orders this thread, the block
        // barrier below the others, and every value written during a sweep
        // is read from L2 (ld.global.cg), never from a stale L1 line
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

__device__ __forceinline__ bool grid_sync(const GridSync &gs, unsigned target) {
    grid_arrive(gs);
    return grid_wait(gs, target);
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_coop(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t st,
                               Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Backward sweep work: a warp task is either nets of at most kBwSmallFanout
// sinks (1, 2 or kBwLanes lanes a net, by fanout) or a piece of kBwPiece
// sinks of a larger net; either way a lane holds kBwPerLane sinks.
constexpr int kBwSmallFanout = 8;
constexpr int kBwLanes = 4;  // lanes of the largest small net
constexpr int kBwPerLane = kBwSmallFanout / kBwLanes;
constexpr int kBwPiece = 32 * kBwPerLane;
constexpr int kBwSplit = 1 << 30;  // on a task's driver pin: the net has several pieces
constexpr int kBwG4 = 1 << 29;     // on a small net's driver pin: the net has 4 lanes
constexpr int kBwG2 = 1 << 28;     // ... 2 lanes (else 1)
constexpr int kBwPinMask = kBwG2 - 1;

// ------------------------------------------------------------ the graph ---
// Device arrays common to both precisions (topology, built once).
struct Topo {
    int32_t n_cells = 0, n_pins = 0, n_nets = 0, n_comb = 0, n_in = 0, n_ep = 0, depth = 0;
    int32_t n_big = 0;
    int32_t *pin_cell = nullptr, *pin_net = nullptr, *net_ptr = nullptr;
    uint8_t *pin_kind = nullptr;
    int32_t *sink_out = nullptr;   // comb input -> its cell's output pin (else -1)
    int32_t *sink_onet = nullptr;  // comb input -> net driven by its cell (else -1)
    int32_t *net_level = nullptr;  // level of the driving cell (0 for FF/PI)
    int32_t *big_nets = nullptr;   // nets with more than kBigFanout sinks
    // combinational cells in level order and their inputs (CSR)
    int32_t *lv_out = nullptr;     // [n_comb] output pin
    int32_t *lv_onet = nullptr;    // [n_comb] net driven by the cell
    int32_t *lv_in_ptr = nullptr;  // [n_comb+1]
    int32_t *lv_in_pin = nullptr;  // [n_in] input pins, ascending
    int32_t *lv_in_drv = nullptr;  // [n_in] driver pin of the input's net
    int32_t *lv_in_net = nullptr;  // [n_in] net of the input
    uint8_t *lv_in_flags = nullptr; // [n_in] kInComb | kInPrev
    // the same, padded for loads in one round: per cell (net driven, output
    // pin, inputs, first input), and kPre input slots per cell
    // (pin, net, driver pin, flags) for cells of at most kPre inputs
    int4 *lv_rec = nullptr;        // [n_comb]
    int4 *lv_slot = nullptr;       // [n_comb * kPre]
    int32_t *ep = nullptr;         // [n_ep] endpoint pins, ascending
    int2 *ep_pd = nullptr;         // [n_ep] (endpoint pin, driver pin of its net)
    int32_t *cp_ptr = nullptr;     // [n_cells+1] cell -> pins CSR
    int32_t *cp = nullptr;         // [n_pins]
    int32_t *slot_of_pin = nullptr;// [n_pins] position of a pin in cp
    uint8_t *cell_fixed = nullptr; // [n_cells]
    // backward sweep warp tasks, deepest level first: per task and lane the
    // net's driver pin (| kBwSplit) and the net, and kBwPerLane sink slots
    // (pin, kind | kKindPrev, net driven by the sink's cell; pin -1: none)
    int2 *bw_drv = nullptr;  // [n_bw_tasks * 32]
    int4 *bw_slot = nullptr; // [n_bw_tasks * 32 * kBwPerLane]
    int32_t n_bw_tasks = 0;
    // device copies of the level structure for the single-launch sweeps:
    // lvl_ptr [depth+1] as in Levels, bw_lv [depth+1] = (first task,
    // small-net tasks, piece tasks, 0) of each level
    int32_t *lvl_ptr = nullptr;
    int4 *bw_lv = nullptr;
};

// Incremental propagation (sta_propagate_incremental).  Every array is
// indexed by net; a stamp equal to `cur` (the number of the current
// incremental call) marks the net for this call only, so nothing is cleared
// between calls.
struct Inc {
    int32_t *stamp = nullptr;   // a cell on the net moved, or its driver's outputs changed
    int2 *span = nullptr;       // (lo, hi): levels of the cells a change of the net reaches
                                // (its driving cell when combinational, its sinks' cells)
    int2 *cspan = nullptr;      // [n_cells] the spans of a cell's nets, combined
    // [3] levels the changes of this call reach; the level after which they
    // saturated, plus one (INT_MAX: they did not)
    int32_t *lohi = nullptr;
    int32_t *lvchg = nullptr;   // [depth + 2] cells whose outputs changed, per level
    // [3] moved cells, cells re-evaluated selectively, of them cells with
    // changed outputs
    unsigned long long *cnt = nullptr;
    int cur = 0;
};

// Host copies of the launch structure of the level sweeps.
struct Levels {
    std::vector<int32_t> lvl_ptr;   // comb cells of level l: [lvl_ptr[l-1], lvl_ptr[l])
    // backward sweep of level l: small-net tasks [bw_s_lo[l], +bw_s_n[l]),
    // then pieces of larger nets [bw_b_lo[l], +bw_b_n[l])
    std::vector<int32_t> bw_s_lo, bw_s_n, bw_b_lo, bw_b_n;
};

// Nodes of the report_timing(n) prefix tree, one path each (structure of
// arrays): parent node (-1 for an endpoint's worst path), the sidetrack pin
// that the node adds to its parent (-1: none), endpoint, pins on the path,
// sidetracks on the path, cost (slack gained over the endpoint's worst path)
// and the order-preserving bits of the path slack.
template <typename R>
struct RtNodes {
    int32_t *par = nullptr, *side = nullptr, *ep = nullptr, *len = nullptr, *nsd = nullptr;
    R *cost = nullptr;
    unsigned long long *key = nullptr;
};

template <typename R>
struct State {
    using A = typename Acc<R>::T;
    R *pin_dx = nullptr, *pin_dy = nullptr, *pin_cap = nullptr, *cell_rdrv = nullptr;
    R *tnet = nullptr;    // [n_pins]
    R *cload = nullptr;   // [n_nets]
    R *dnet = nullptr;    // [n_nets] delay of the driving cell
    A *arr = nullptr, *req = nullptr;  // [n_pins]
    R *slack = nullptr;   // [n_pins]
    int2 *pred = nullptr;         // [n_nets] worst input pin of the driving cell (-1: startpoint), its net
    int32_t *plen = nullptr;      // [n_nets] pins from the driver back to its startpoint
    double *T = nullptr;          // device clock period
    unsigned *gsync = nullptr;    // [4] forward barrier count, sticky timeout status, backward barrier count
    double *wns_tns = nullptr;    // [2]
    double *red_part = nullptr;   // [2 * chunks] WNS / TNS partials per kRedChunk endpoints
    unsigned *red_count = nullptr;
    // [n_nets] required time of each net's driver during the backward sweep,
    // as an order-preserving integer key (pieces of a net combine by atomicMin)
    unsigned long long *reqkey = nullptr;
    // extraction
    uint64_t *sort_a = nullptr, *sort_b = nullptr;  // (key, pin) items, ping-pong
    int32_t *nviol = nullptr;     // device count of failing endpoints
    int32_t *viol = nullptr;      // [n_ep] failing endpoints, by (slack, pin) or by pin (see viol_sorted)
    uint8_t *ep_flag = nullptr;   // [n_ep + 32] endpoint fails
    BEnt<R> *blist = nullptr;     // [n_nets * kMaxK] sidetrack lists, list_group(list_L) apart
    int32_t *bcnt = nullptr;      // [n_nets] entries in each sidetrack list
    int32_t *p_parent = nullptr, *p_side = nullptr, *p_len = nullptr;  // [n_ep * K]
    R *p_cost = nullptr;
    int32_t *p_count = nullptr;   // [n_ep] paths per failing endpoint (sorted order)
    long long *n_paths = nullptr; // device total
    // pin pairs
    long long *sumq = nullptr, *maxq = nullptr;  // [n_pins] fixed-point slack/WNS
    uint8_t *in_p = nullptr;   // [n_pins]
    R *w = nullptr;                               // [n_pins]
    long long *n_pairs = nullptr;
    // pairs, compacted for the loss: the sink pins of P, and the cells with
    // a pin in a pair (its sink or the driver of its net); the lists are
    // ascending, counts in pcnt[0] (pins) and pcnt[1] (cells).  cell_pf
    // flags those cells, net_pf the nets holding a sink of P
    uint8_t *net_pf = nullptr;    // [n_nets] 0, kPfSmall or kPfLarge
    uint8_t *cell_pf = nullptr;   // [n_cells]
    int32_t *ppins = nullptr;     // [n_pins]
    int32_t *pcells = nullptr;    // [n_cells]
    int32_t *pcnt = nullptr;      // [2]
    // stream compaction (compact_u8): a state word per tile of flags and two
    // counters (tiles taken, blocks done)
    unsigned long long *cmp_tiles = nullptr;
    unsigned *cmp_ctr = nullptr;
    // pair records, one per sink of P in the order of ppins, rebuilt after
    // every change of P: (sink's cell, driver's cell, sink's gradient slot,
    // driver's gradient slot for the first pair of a net of at most
    // kBigFanout sinks, else -1); pin offsets (sink x, y, driver x, y); the
    // weight; for a net's first pair, the net's pairs.  pr_big lists the
    // nets of more than kBigFanout sinks holding a pair: (first record,
    // pairs, driver's gradient slot, 0), pr_nbig of them
    int4 *pr_a = nullptr;         // [n_sinks]
    R *pr_o = nullptr;            // [4 * n_sinks]
    R *pr_w = nullptr;            // [n_sinks]
    int32_t *pr_n = nullptr;      // [n_sinks]
    int4 *pr_big = nullptr;       // [n_big]
    int32_t *pr_nbig = nullptr;
    // loss
    R *gslot = nullptr;           // [2*n_pins] pin gradients in cell-slot order (x, y); zero outside P
    double *loss_part = nullptr;
    unsigned *loss_count = nullptr;
    // report_timing(n): the kept prefix-tree nodes, the report (node indices,
    // worst first) and each reported path's sidetracks, deepest first, at
    // rt_side_off[q] (grown on demand, freed by rt_free)
    RtNodes<R> rt;
    // per report, from the last propagation: per net driven by a
    // combinational cell (next net on its worst-input chain, first input in
    // lv_in order, inputs, worst input pin; all -1 elsewhere), and per input
    // the slack a sidetrack through it costs
    int4 *rt_chain = nullptr;
    R *rt_delta = nullptr;
    // incremental propagation: cell positions of the last propagation
    R *xprev = nullptr, *yprev = nullptr;
    // net weighting (net_weights_update): a weight per net, and the count of
    // nets with negative slack of the last update
    R *net_w = nullptr;
    int32_t *n_crit = nullptr;
    int32_t *rt_out = nullptr;
    int64_t *rt_side_off = nullptr;
    int32_t *rt_sides = nullptr;
};

}  // namespace tdp

struct tdp_graph {
    tdp_precision prec = TDP_FP32;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;  // stream used to capture CUDA graphs
    // the backward sweep runs on `side` once the graph's stream reaches
    // ev_bwd_go (the end of the forward sweep); ev_bwd marks its end,
    // bwd_pending until the graph's stream waits for it
    cudaStream_t side = nullptr;
    cudaEvent_t ev_bwd_go = nullptr, ev_bwd = nullptr;
    bool overlap_bwd = true, bwd_pending = false;
    // the overlapped backward sweep's share of its resident grid, in 16ths
    // (TDP_BWD_SHARE at sta_build, 1 to 16)
    int bwd_share = 9;
    // a full propagation starts the backward sweep right after net RC on
    // bwd_sms blocks (one an SM) and runs the forward sweep on the other SMs
    // (0: chosen by bwd_split at the first propagation; TDP_BWD_SMS at
    // sta_build sets it, a negative value there: the backward sweep after
    // the forward sweep, beside the rest, as incremental propagation runs it)
    int bwd_sms = 0;
    unsigned cmp_epoch = 0;  // calls of the single-pass compaction (its tile states' tag)
    tdp::Topo topo;
    tdp::Levels lv;
    tdp::State<float> s32;
    tdp::State<double> s64;
    double r = 0, c = 0, d0 = 0;
    int K = 0, keep_nonneg = 0, n_endpoints = -1;
    int loss_kind = 0;  // tdp_loss_kind of the attraction loss
    bool net_w_init = false;  // net weights allocated and set to 1
    bool propagated = false, extracted = false;
    // failing endpoints: sorted by (slack, pin), or (extraction of all of
    // them) by pin until sta_get_paths sorts them and their path records
    bool viol_sorted = true;
    // sidetrack lists are built by the forward sweep: list_L entries per node
    // (the K - 1 of the last extraction), lists_valid_L of them are current
    int list_L = 0, lists_valid_L = 0;
    // the last extraction was report_timing(n): rt_n_out paths in the rt
    // buffers of the state (else report_timing_endpoint's per-endpoint records)
    bool rt_mode = false;
    int64_t rt_n_out = 0, rt_n_sides = 0;
    int64_t rt_cap = 0, rt_out_cap = 0, rt_soff_cap = 0, rt_sides_cap = 0;  // buffer capacities
    int rt_rounds = 0;                                     // expansion rounds of the last report
    // incremental propagation: inc_valid while the state holds the timing of
    // the positions in xprev / yprev; inc_full when the last incremental call
    // re-timed everything
    tdp::Inc inc;
    bool inc_valid = false, inc_full = true;
    int64_t rt_nodes = 0;                                  // nodes the last report kept
    // level sweeps: one cooperative launch each (single_launch), else CUDA
    // graphs of one kernel per level
    bool single_launch = true;
    int n_sm = 0;
    std::vector<std::pair<const void *, int>> coop_grid;  // kernel -> resident grid
    cudaGraphExec_t fwd_graph = nullptr, bwd_graph = nullptr;  // captured level sweeps
    int fwd_graph_L = -1, fwd_graph_kernels = 0, bwd_graph_kernels = 0;
    std::vector<void *> allocs;  // every device allocation, freed in sta_destroy
    // instrumentation
    int64_t n_launch = 0;                 // kernels queued by this graph so far
    int prof_id = -1;                     // kernel timed with CUDA events (-1: none)
    std::vector<cudaEvent_t> prof_free;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_pending;
};

namespace tdp {
// Every device allocation of the library goes through dalloc (cudaMalloc,
// owned by the graph) or dmalloc_async (cudaMallocAsync, temporaries).  The
// test hook tdp_debug_fail_alloc can make one of them fail on the host
// without calling CUDA, so that the out-of-memory paths are tested without
// exhausting a GPU.
bool alloc_fail_injected();
template <typename T>
cudaError_t dmalloc_async(T **p, size_t bytes, cudaStream_t st) {
    if (alloc_fail_injected()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocAsync(p, bytes, st);
}

template <typename T>
tdp_status dalloc(tdp_graph *g, T **p, size_t n) {
    void *q = nullptr;
    size_t bytes = n * sizeof(T);
    if (bytes == 0) bytes = sizeof(T);
    cudaError_t e = alloc_fail_injected() ? cudaErrorMemoryAllocation : cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        return TDP_ERR_OOM;
    }
    g->allocs.push_back(q);
    *p = static_cast<T *>(q);
    return TDP_OK;
}

template <typename R>
State<R> &state(tdp_graph *g);
template <>
inline State<float> &state<float>(tdp_graph *g) { return g->s32; }
template <>
inline State<double> &state<double>(tdp_graph *g) { return g->s64; }

template <typename R>
tdp_status propagate_impl(tdp_graph *g, const R *x, const R *y, double T);
// the forward sweep building the lists; leave_sms: SMs to leave to a
// backward sweep that runs at the same time (single launch); after_rc: net RC
// is the stream's last kernel and has zeroed the sweep's barrier word
template <typename R>
tdp_status forward_lists(tdp_graph *g, int leave_sms = 0, bool after_rc = false);
template <typename R>
tdp_status extract_impl(tdp_graph *g, int n_endpoints, int K, int keep_nonneg);
template <typename R>
tdp_status get_paths_impl(tdp_graph *g, int32_t *viol, int32_t *ep, R *slack, int64_t *pin_ptr,
                          int32_t *pins);
template <typename R>
tdp_status update_pairs_impl(tdp_graph *g, double w0, double w1);
template <typename R>
tdp_status report_impl(tdp_graph *g, int64_t n, int keep_nonneg);
template <typename R>
tdp_status rt_get_paths(tdp_graph *g, int32_t *ep, R *slack, int64_t *pin_ptr, int32_t *pins);
template <typename R>
tdp_status rt_paths_size(tdp_graph *g, int64_t *npin_out);
// the pair update's walk over the reported paths (report_timing mode)
template <typename R>
void rt_pair_walk(tdp_graph *g);
// frees the report_timing buffers of both states
void rt_free(tdp_graph *g);

// failing endpoints sorted by (slack, pin) into viol / nviol of the state
template <typename R>
tdp_status sort_failing(tdp_graph *g);

// (key, index) items; sort_items sorts the first *count (at most n) of a by
// (key, pin) and leaves the result in a (a and b are swapped as needed)
struct SortItem {
    unsigned long long key;  // order-preserving bits of a value
    unsigned long long pin;
};
void sort_items(SortItem *&a, SortItem *&b, const int *count, int n, cudaStream_t st);

// Walk one extracted path from its endpoint back to its startpoint, calling
// visit(pin, is_sink) for every pin in that order.  The path leaves the
// worst-input chain at its sidetracks, sides[nsides - 1] (nearest the
// endpoint) first, sides[0] (deepest) last.
template <typename R, typename F>
__device__ __forceinline__ void walk_path(const Topo &t, const State<R> &s, int ep, const int *sides,
                                          int nsides, F &&visit) {
    visit(ep, true);
    int e = t.pin_net[ep];
    int j = nsides - 1;
    for (;;) {
        visit(t.net_ptr[e], false);
        const int2 pr = s.pred[e];
        int pi = pr.x;
        if (pi < 0) break;
        int nx;
        if (j >= 0 && t.sink_onet[sides[j]] == e) {
            pi = sides[j--];
            nx = t.pin_net[pi];
        } else {
            nx = pr.y;
        }
        visit(pi, true);
        e = nx;
    }
}
template <typename R>
tdp_status loss_fwd_impl(tdp_graph *g, const R *x, const R *y, double beta, double *loss);
template <typename R>
tdp_status loss_bwd_impl(tdp_graph *g, const R *x, const R *y, double beta, const double *gs,
                         R *gx, R *gy);

// reads and clears the sticky status of the grid barriers (synchronises the
// stream); TDP_ERR_TIMEOUT if a wait gave up since the last check
tdp_status check_sync_status(tdp_graph *g);

// one flag array of a stream compaction: the indices i < n (or map[i]) with
// f[i] == val, ascending, go to out and their number to the device word
// count
struct CmpPart {
    const uint8_t *f;
    const int32_t *map;
    int32_t *out;
    int32_t *count;
    int n;
    uint8_t val;
};

// the compaction of one flag array (b == nullptr) or of two in one launch
// (flags padded to a multiple of 32 bytes); the launch also sets the device
// words clear32 and clear64 to 0 where given (counters of the kernels after
// it, so that the stream needs no memset between them).  Launched as a
// programmatic dependent of the kernel before it (launch_pdl, chain_enter).
tdp_status compact_flags(tdp_graph *g, const CmpPart &a, const CmpPart *b = nullptr, int32_t *clear32 = nullptr,
                         long long *clear64 = nullptr);
inline tdp_status compact_u8(tdp_graph *g, const uint8_t *flags, uint8_t val, int n, const int32_t *map,
                             int32_t *out, int32_t *count) {
    return compact_flags(g, CmpPart{flags, map, out, count, n, val});
}

// tile states the compaction of the graph's largest flag arrays needs
inline size_t compact_tile_cap(const Topo &t) {
    return (size_t)std::max(t.n_pins + t.n_cells, t.n_nets) / kCompactItems + 4;
}

// rebuild the compacted pair lists (ppins, pcells, pcnt) from in_p / cell_pf
template <typename R>
tdp_status compact_pairs(tdp_graph *g);

// exclusive scan of n int32 counts into int64 offsets (out has n+1 entries)
tdp_status scan_i32_to_i64(tdp_graph *g, const int32_t *in, int64_t *out, int64_t n,
                           cudaStream_t st);

inline int div_up(int64_t a, int64_t b) { return static_cast<int>((a + b - 1) / b); }

// Lanes per cell in the forward sweep for sidetrack lists of L entries,
// which is also the stride (in entries) between two nets' lists.
__host__ __device__ constexpr int list_group(int L) { return L == 0 ? 4 : L + 1; }

__device__ __forceinline__ int div_up_dev(int a, int b) { return (a + b - 1) / b; }

// Sidetrack list lengths the forward sweep builds (one kernel each): the
// smallest that holds `need` entries.
inline int list_bucket(int need) {
    const int lens[] = {0, 3, 7, 15, 31};
    for (int l : lens)
        if (l >= need) return l;
    return kMaxK - 1;
}

// Brackets the launches of one kernel with CUDA events on the graph's stream
// when that kernel is selected by tdp_profile_kernel; counts launches always.
struct LaunchScope {
    tdp_graph *g;
    bool on;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    LaunchScope(tdp_graph *g_, KernelId id, int n_kernels = 1, cudaStream_t st_ = nullptr);
    ~LaunchScope();
};

// the graph's stream waits for the last backward sweep (no-op if it already does)
void join_side(tdp_graph *g);
}  // namespace tdp
