// Static timing analysis on the device (Section II-B; Eq. (2) slack;
// Eqs. (3)-(4) WNS/TNS; Eq. (8) Elmore net delay).
//
//   k_net_rc     one pass over the nets: pin positions, Elmore delay of every
//                sink, net load and driving-cell delay (thread per net up to 32
//                sinks, block per net above, FP64 load sum there)
//   k_fwd_level  arrival times of the combinational cells of one level (thread
//                per cell; max / argmax over its inputs), and, when asked, the
//                cell's sidetrack list for report_timing_endpoint
//   k_bwd_level  required times of the nets driven from one level (lane per
//                net of at most 8 sinks, warp per 128 sinks of larger nets,
//                split nets combined by the last warp to finish)
//   k_wns_tns    FP64 WNS / TNS over the endpoints (fixed-order reduction)
//
// The per-level launches are captured once into a CUDA graph and replayed.
// Every array a level kernel reads was written by an earlier launch (a lower
// level going forward, a higher level going backward), so the reads use the
// read-only path and all loads of a group of inputs / sinks are issued before
// the first store.
#include <type_traits>

#include "tdp_internal.cuh"

namespace tdp {

template <typename R>
__device__ __forceinline__ typename Acc<R>::T acc_from_double(double v);
template <>
__device__ __forceinline__ double acc_from_double<double>(double v) { return v; }
template <>
__device__ __forceinline__ fx2 acc_from_double<float>(double v) {
    float hi = (float)v;
    return fx2{hi, (float)(v - (double)hi)};
}

// ------------------------------------------------------------- net RC ---

template <typename R>
__device__ __forceinline__ void net_finish(const Topo &t, State<R> &s, int e, int drv, int cd,
                                           double load, R d0) {
    R ld = (R)load;
    s.cload[e] = ld;
    R dd = d0 + ldg(&s.cell_rdrv[cd]) * ld;
    s.dnet[e] = dd;
    if (ldg(&t.pin_kind[drv]) == PK_START) s.arr[drv] = Acc<R>::make(dd);
}

// Elmore delay of the sinks first, first+step, ... < b of the net driven by
// pin a (Eq. (8)); returns the part of the net's load they contribute.
template <typename R>
__device__ __forceinline__ double sinks_rc(const Topo &t, State<R> &s, const R *x, const R *y,
                                           int a, int b, int first, int step, R r, R c) {
    const int cd = ldg(&t.pin_cell[a]);
    const R xd = ldg(&x[cd]) + ldg(&s.pin_dx[a]), yd = ldg(&y[cd]) + ldg(&s.pin_dy[a]);
    double load = 0.0;
#pragma unroll 4
    for (int p = first; p < b; p += step) {
        const int cs = ldg(&t.pin_cell[p]);
        const R L = fabs(ldg(&x[cs]) + ldg(&s.pin_dx[p]) - xd) + fabs(ldg(&y[cs]) + ldg(&s.pin_dy[p]) - yd);
        const R Rw = r * L, Cw = c * L;
        const R cap = ldg(&s.pin_cap[p]);
        s.tnet[p] = Rw * (Cw * R(0.5) + cap);
        load += (double)(Cw + cap);
    }
    return load;
}

constexpr int kRcThreads = 256;

// Blocks [0, n_small_blocks): one thread per net with at most kBigFanout sinks.
// Blocks after that: one block per high-fanout net (FP64 load sum, fixed order).
template <typename R>
__global__ void __launch_bounds__(kRcThreads) k_net_rc(Topo t, State<R> s, const R *__restrict__ x,
                                                       const R *__restrict__ y, double T, R r, R c,
                                                       R d0, int n_small_blocks) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *s.T = T;
    if ((int)blockIdx.x < n_small_blocks) {
        const int e = blockIdx.x * kRcThreads + threadIdx.x;
        if (e >= t.n_nets) return;
        const int a = ldg(&t.net_ptr[e]), b = ldg(&t.net_ptr[e + 1]);
        if (b - a - 1 > kBigFanout) return;
        // FP32 sum for nets of at most kBigFanout sinks
        const int cd = ldg(&t.pin_cell[a]);
        const R xd = ldg(&x[cd]) + ldg(&s.pin_dx[a]), yd = ldg(&y[cd]) + ldg(&s.pin_dy[a]);
        R load = 0;
#pragma unroll 4
        for (int p = a + 1; p < b; ++p) {
            const int cs = ldg(&t.pin_cell[p]);
            const R L = fabs(ldg(&x[cs]) + ldg(&s.pin_dx[p]) - xd) + fabs(ldg(&y[cs]) + ldg(&s.pin_dy[p]) - yd);
            const R Rw = r * L, Cw = c * L;
            const R cap = ldg(&s.pin_cap[p]);
            s.tnet[p] = Rw * (Cw * R(0.5) + cap);
            load += Cw + cap;
        }
        net_finish(t, s, e, a, cd, (double)load, d0);
        return;
    }
    __shared__ double part[kRcThreads / 32];
    const int e = ldg(&t.big_nets[blockIdx.x - n_small_blocks]);
    const int a = ldg(&t.net_ptr[e]), b = ldg(&t.net_ptr[e + 1]);
    double load = sinks_rc<R>(t, s, x, y, a, b, a + 1 + threadIdx.x, kRcThreads, r, c);
    for (int o = 16; o > 0; o >>= 1) load += __shfl_xor_sync(0xffffffffu, load, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = load;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int k = 0; k < kRcThreads / 32; ++k) tot += part[k];
        net_finish(t, s, e, a, ldg(&t.pin_cell[a]), tot, d0);
    }
}

// ------------------------------------------------------------ forward ---

constexpr int kLvThreads = 128;

// A list entry while a list is being built: the deviation cost and a key that
// orders equal costs.  key = (group << 29) | pin, group 0 for the node's own
// deviations through a pin below its worst input, 1 for inherited entries, 2
// for own deviations through a pin above the worst input.  Own entries are
// only ever compared with entries of other groups or with own entries, so the
// pins of inherited entries never decide an order.
template <typename R>
struct LEnt {
    R d;
    uint32_t key;
};
constexpr uint32_t kPinMask = (1u << 29) - 1u;
constexpr uint32_t kNoneKey = 0xffffffffu;

template <typename R>
__device__ __forceinline__ bool lent_before(const LEnt<R> &a, const LEnt<R> &b) {
    return a.d < b.d || (a.d == b.d && a.key < b.key);
}

template <typename R>
__device__ __forceinline__ R r_inf() {
    return (R)__longlong_as_double(0x7ff0000000000000ll);
}

// Sidetrack list of one node (Section III-B extraction): the L cheapest
// deviations on the worst-input chain from the node back to its startpoint.
// A deviation enters a node through an input other than its worst one; its
// cost is Arr(worst input) - Arr(that input).  The list is the node's own
// deviations merged into the list of its worst input's driver; equal costs
// are ordered as the resulting paths' pin sequences (read from the endpoint)
// would be: own deviations through a pin below the worst input, then the
// inherited entries, then own deviations through a pin above it.  Lists hold
// exactly L entries; unused ones are +inf sentinels (pin -1).
template <typename R, int L, int NIN>
__device__ __forceinline__ void build_list(State<R> &s, int e, int bi, int bn, bool bn_comb,
                                           typename Acc<R>::T best, const int *ip,
                                           const typename Acc<R>::T *ain, int nin) {
    using AC = Acc<R>;
    LEnt<R> li[L];
    if (bn_comb) {  // the inherited list (written by an earlier level's launch)
        const BEnt<R> *src = s.blist + (size_t)bn * L;
#pragma unroll
        for (int j = 0; j < L; ++j) {
            const BEnt<R> v = ldg(&src[j]);
            li[j] = LEnt<R>{v.delta, v.pin < 0 ? kNoneKey : ((1u << 29) | (uint32_t)v.pin)};
        }
    } else {
#pragma unroll
        for (int j = 0; j < L; ++j) li[j] = LEnt<R>{r_inf<R>(), kNoneKey};
    }
#pragma unroll
    for (int u = 0; u < NIN; ++u) {
        if (u >= nin || ip[u] == bi) continue;
        const LEnt<R> x{AC::diff(best, ain[u]), ((ip[u] < bi ? 0u : 2u) << 29) | (uint32_t)ip[u]};
        // insert x, keeping the first L entries (compare-and-shift from the top)
#pragma unroll
        for (int j = L - 1; j >= 0; --j) {
            const bool shift = j > 0 && lent_before(x, li[j - 1]);
            const bool here = lent_before(x, li[j]);
            li[j] = shift ? li[j - 1] : (here ? x : li[j]);
        }
    }
    BEnt<R> *out = s.blist + (size_t)e * L;
    int m = 0;
#pragma unroll
    for (int j = 0; j < L; ++j) {
        const bool none = li[j].key == kNoneKey;
        out[j] = BEnt<R>{li[j].d, none ? -1 : (int32_t)(li[j].key & kPinMask)};
        m += none ? 0 : 1;
    }
    s.bcnt[e] = m;
}

// Arrival of one combinational cell (k in level order) whose inputs are
// [a, b) with b - a <= NIN; builds its sidetrack list when L > 0.
template <typename R, int L, int NIN>
__device__ __forceinline__ void fwd_cell(const Topo &t, State<R> &s, int k, int a, int b) {
    using AC = Acc<R>;
    using A = typename AC::T;
    const int e = ldg(&t.lv_onet[k]), o = ldg(&t.lv_out[k]);
    int ip[NIN], in[NIN], dv[NIN], pl[NIN];
    uint8_t cb[NIN];
    A av[NIN];
    R tv[NIN];
    // every load of the cell's inputs first, then the arithmetic, then stores
#pragma unroll
    for (int u = 0; u < NIN; ++u) {
        if (a + u < b) {
            ip[u] = ldg(&t.lv_in_pin[a + u]);
            in[u] = ldg(&t.lv_in_net[a + u]);
            dv[u] = ldg(&t.lv_in_drv[a + u]);
            cb[u] = ldg(&t.lv_in_comb[a + u]);
        }
    }
    pdl_wait();  // everything below reads values earlier kernels wrote
    const R dcell = ldg(&s.dnet[e]);
#pragma unroll
    for (int u = 0; u < NIN; ++u) {
        if (a + u < b) {
            av[u] = ldg(&s.arr[dv[u]]);
            tv[u] = ldg(&s.tnet[ip[u]]);
            pl[u] = ldg(&s.plen[in[u]]);
        }
    }
    // inputs ascending by pin: strict > keeps the lowest pin on ties (and the
    // first input if arrivals are not comparable)
    int bi = -1, bn = -1, bl = 0;
    bool bc = false;
    A best = AC::ninf();
#pragma unroll
    for (int u = 0; u < NIN; ++u) {
        if (a + u < b) {
            av[u] = AC::add(av[u], tv[u]);
            if (bi < 0 || AC::gt(av[u], best)) {
                best = av[u];
                bi = ip[u];
                bn = in[u];
                bl = pl[u];
                bc = cb[u];
            }
        }
    }
#pragma unroll
    for (int u = 0; u < NIN; ++u)
        if (a + u < b) s.arr[ip[u]] = av[u];
    s.arr[o] = AC::add(best, dcell);
    s.pred_in[e] = bi;
    s.pred_net[e] = bn;
    s.plen[e] = bl + 2;
    if constexpr (L > 0) build_list<R, L, NIN>(s, e, bi, bn, bc, best, ip, av, b - a);
}

template <typename R, int L>
__global__ void __launch_bounds__(kLvThreads) k_fwd_level(Topo t, State<R> s, int lo, int hi) {
    pdl_trigger();
    const int k = lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= hi) return;
    const int a = ldg(&t.lv_in_ptr[k]), b = ldg(&t.lv_in_ptr[k + 1]);
    if (b - a <= kPre) fwd_cell<R, L, kPre>(t, s, k, a, b);
    else fwd_cell<R, L, kMaxFanin>(t, s, k, a, b);
}

template <typename R>
static void launch_fwd(const Topo &t, const State<R> &s, int lo, int hi, int L, cudaStream_t cs) {
    const int grid = div_up(hi - lo, kLvThreads);
    switch (L) {
        case 0: launch_pdl(k_fwd_level<R, 0>, grid, kLvThreads, cs, t, s, lo, hi); break;
        case 3: launch_pdl(k_fwd_level<R, 3>, grid, kLvThreads, cs, t, s, lo, hi); break;
        case 7: launch_pdl(k_fwd_level<R, 7>, grid, kLvThreads, cs, t, s, lo, hi); break;
        case 15: launch_pdl(k_fwd_level<R, 15>, grid, kLvThreads, cs, t, s, lo, hi); break;
        default: launch_pdl(k_fwd_level<R, 31>, grid, kLvThreads, cs, t, s, lo, hi); break;
    }
}

// ----------------------------------------------------------- backward ---

// req / slack of the sinks first, first+step, ... < b of the net driven by
// pin a, NP sinks per round of loads; returns min over them of req(s) - t(s)
// and the driver's arrival in ad.  The first round's topology loads are
// issued before pdl_wait().
template <typename R, int NP>
__device__ __forceinline__ typename Acc<R>::T net_sinks_req(const Topo &t, State<R> &s, int first,
                                                            int b, int step, int a,
                                                            typename Acc<R>::T &ad) {
    using AC = Acc<R>;
    using A = typename AC::T;
    A m = AC::pinf();
    uint8_t kd[NP];
    int so[NP], sn[NP];
    auto topo_loads = [&](int p0) {
#pragma unroll
        for (int u = 0; u < NP; ++u) {
            const int p = p0 + u * step;
            if (p < b) {
                kd[u] = ldg(&t.pin_kind[p]);
                so[u] = ldg(&t.sink_out[p]);
                sn[u] = ldg(&t.sink_onet[p]);
            }
        }
    };
    topo_loads(first);
    pdl_wait();  // everything below reads values earlier kernels wrote
    ad = ldg(&s.arr[a]);
    const A Tacc = acc_from_double<R>(*s.T);
    for (int p0 = first; p0 < b; p0 += NP * step) {
        if (p0 != first) topo_loads(p0);
        R tp[NP];
#pragma unroll
        for (int u = 0; u < NP; ++u) {
            const int p = p0 + u * step;
            if (p < b) tp[u] = ldg(&s.tnet[p]);
        }
        A rq[NP], ap[NP];
#pragma unroll
        for (int u = 0; u < NP; ++u) {
            const int p = p0 + u * step;
            if (p < b) {
                if (kd[u] == PK_ENDPOINT) {
                    ap[u] = AC::add(ad, tp[u]);
                    rq[u] = Tacc;
                } else {
                    rq[u] = AC::add(ldg(&s.req[so[u]]), -ldg(&s.dnet[sn[u]]));
                    ap[u] = ldg(&s.arr[p]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < NP; ++u) {
            const int p = p0 + u * step;
            if (p < b) {
                if (kd[u] == PK_ENDPOINT) s.arr[p] = ap[u];
                s.req[p] = rq[u];
                s.slack[p] = AC::diff(rq[u], ap[u]);
                const A cand = AC::add(rq[u], -tp[u]);
                if (AC::lt(cand, m)) m = cand;
            }
        }
    }
    return m;
}

template <typename A>
__device__ __forceinline__ A shfl_xor_acc(A v, int o) {
    if constexpr (std::is_same<A, double>::value) {
        return __shfl_xor_sync(0xffffffffu, v, o);
    } else {
        A r;
        r.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        r.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        return r;
    }
}

// L2 loads of values another block of the same launch has just written.
__device__ __forceinline__ double ldcg_acc(const double *p) { return __ldcg(p); }
__device__ __forceinline__ fx2 ldcg_acc(const fx2 *p) {
    float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
    return fx2{v.x, v.y};
}

// One warp per task of this level: warps [0, ns) take groups s_lo.. of 32
// small nets (a lane per net, all its sinks in one round of loads), warps
// [ns, ns + nb) take pieces b_lo.. of larger nets (lanes stride the sinks).
template <typename R>
__global__ void __launch_bounds__(kLvThreads) k_bwd_level(Topo t, State<R> s, int s_lo, int ns,
                                                          int b_lo, int nb) {
    using AC = Acc<R>;
    using A = typename AC::T;
    pdl_trigger();
    const int w = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (w < ns) {
        const int i = (s_lo + w) * 32 + lane;
        const int a = ldg(&t.bw_sa[i]), b = ldg(&t.bw_sb[i]);
        if (a < 0) return;
        A ad;
        const A m = net_sinks_req<R, kBwSmallFanout>(t, s, a + 1, b, 1, a, ad);
        s.req[a] = m;
        s.slack[a] = AC::diff(m, ad);
        return;
    }
    if (w >= ns + nb) return;
    const BwTask task = t.bw_task[b_lo + (w - ns)];
    const int a = task.drv;
    A ad;
    A m = net_sinks_req<R, kPre>(t, s, task.p0 + lane, task.p1, 32, a, ad);
    for (int o = 16; o > 0; o >>= 1) {  // min is exact: any order gives the same value
        const A other = shfl_xor_acc(m, o);
        if (AC::lt(other, m)) m = other;
    }
    if (lane != 0) return;
    if (task.nparts > 1) {
        // several warps share this net: each leaves its minimum in a slot,
        // and the last one to finish combines them (the counter only grows)
        s.bw_part[task.slot] = m;
        __threadfence();
        const unsigned long long done = atomicAdd(&s.bw_cnt[task.cnt], 1ull) + 1ull;
        if (done % (unsigned long long)task.nparts != 0ull) return;
        __threadfence();
        const int base = task.slot - task.part;
        m = ldcg_acc(&s.bw_part[base]);
        for (int j = 1; j < task.nparts; ++j) {
            const A v = ldcg_acc(&s.bw_part[base + j]);
            if (AC::lt(v, m)) m = v;
        }
    }
    s.req[a] = m;
    s.slack[a] = AC::diff(m, ad);
}

// ---------------------------------------------------------- WNS / TNS ---

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 148;

// WNS = min over endpoints with negative slack, TNS = their sum (FP64).
// Each block reduces a fixed stride of endpoints; the last block to finish
// combines the per-block partials in block order, so the result does not
// depend on scheduling.
template <typename R>
__global__ void __launch_bounds__(kRedThreads) k_wns_tns(Topo t, State<R> s) {
    __shared__ double smin[kRedThreads / 32], ssum[kRedThreads / 32];
    __shared__ bool last;
    pdl_wait();
    double mn = 0.0, sm = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < t.n_ep; i += gridDim.x * blockDim.x) {
        double v = (double)s.slack[t.ep[i]];
        if (v < 0.0) {
            mn = fmin(mn, v);
            sm += v;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        sm += __shfl_xor_sync(0xffffffffu, sm, o);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        smin[w] = mn;
        ssum[w] = sm;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double bm = smin[0], bs = ssum[0];
        for (int k = 1; k < kRedThreads / 32; ++k) {
            bm = fmin(bm, smin[k]);
            bs += ssum[k];
        }
        s.red_part[2 * blockIdx.x] = bm;
        s.red_part[2 * blockIdx.x + 1] = bs;
        __threadfence();
        unsigned ticket = atomicAdd(s.red_count, 1u);
        last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        const volatile double *part = s.red_part;
        double bm = 0.0, bs = 0.0;
        for (int k = 0; k < (int)gridDim.x; ++k) {
            bm = fmin(bm, part[2 * k]);
            bs += part[2 * k + 1];
        }
        s.wns_tns[0] = bm;
        s.wns_tns[1] = bs;
        *s.red_count = 0u;
    }
}

// ------------------------------------------------------------ launch ---

template <typename R>
static tdp_status capture(tdp_graph *g, cudaGraphExec_t *exec, int *n_kernels, bool fwd, bool bwd,
                          int L) {
    Topo &t = g->topo;
    State<R> &s = state<R>(g);
    cudaStream_t cs = g->cap_stream;
    TDP_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    bool ok = true;
    int nk = 0;
    for (int l = 1; fwd && l <= t.depth && ok; ++l) {
        const int lo = g->lv.lvl_ptr[l - 1], hi = g->lv.lvl_ptr[l];
        if (hi > lo) {
            launch_fwd<R>(t, s, lo, hi, L, cs);
            ++nk;
        }
        ok = cudaGetLastError() == cudaSuccess;
    }
    for (int l = t.depth; bwd && l >= 0 && ok; --l) {
        const int ns = g->lv.bw_s_n[l], nb = g->lv.bw_b_n[l];
        if (ns + nb > 0) {
            launch_pdl(k_bwd_level<R>, div_up((int64_t)(ns + nb) * 32, kLvThreads), kLvThreads, cs, t, s,
                       g->lv.bw_s_lo[l], ns, g->lv.bw_b_lo[l], nb);
            ++nk;
        }
        ok = cudaGetLastError() == cudaSuccess;
    }
    if (bwd && ok) {
        launch_pdl(k_wns_tns<R>, kRedBlocks, kRedThreads, cs, t, s);
        ++nk;
        ok = cudaGetLastError() == cudaSuccess;
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &graph);
    if (!ok || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        set_error("capturing the level sweep failed: %s",
                  cudaGetErrorString(e != cudaSuccess ? e : cudaGetLastError()));
        return TDP_ERR_CUDA;
    }
    e = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        *exec = nullptr;
        set_error("cudaGraphInstantiate failed: %s", cudaGetErrorString(e));
        return TDP_ERR_CUDA;
    }
    *n_kernels = nk;
    return TDP_OK;
}

// Forward sweep (one graph replay), building sidetrack lists of length
// g->list_L (0: none).  Run again, it writes the same arrival times.
template <typename R>
tdp_status forward_lists(tdp_graph *g) {
    State<R> &s = state<R>(g);
    if (g->list_L > 0 && !s.blist) TDP_TRY(dalloc(g, &s.blist, (size_t)g->topo.n_nets * (kMaxK - 1)));
    if (!g->fwd_graph || g->fwd_graph_L != g->list_L) {
        if (g->fwd_graph) cudaGraphExecDestroy(g->fwd_graph);
        g->fwd_graph = nullptr;
        TDP_TRY(capture<R>(g, &g->fwd_graph, &g->fwd_graph_kernels, true, false, g->list_L));
        g->fwd_graph_L = g->list_L;
    }
    LaunchScope ls(g, KID_FWD_SWEEP, g->fwd_graph_kernels);
    TDP_CUDA(cudaGraphLaunch(g->fwd_graph, g->stream));
    return TDP_OK;
}

// Backward sweep and WNS / TNS (one graph replay).
template <typename R>
static tdp_status backward(tdp_graph *g) {
    if (!g->bwd_graph) TDP_TRY(capture<R>(g, &g->bwd_graph, &g->bwd_graph_kernels, false, true, 0));
    LaunchScope ls(g, KID_BWD_SWEEP, g->bwd_graph_kernels);
    TDP_CUDA(cudaGraphLaunch(g->bwd_graph, g->stream));
    return TDP_OK;
}

template <typename R>
static tdp_status sweep(tdp_graph *g) {
    TDP_TRY(forward_lists<R>(g));
    return backward<R>(g);
}

template tdp_status forward_lists<float>(tdp_graph *);
template tdp_status forward_lists<double>(tdp_graph *);

template <typename R>
tdp_status propagate_impl(tdp_graph *g, const R *x, const R *y, double T) {
    Topo &t = g->topo;
    State<R> &s = state<R>(g);
    const int nsb = div_up(t.n_nets, kRcThreads);
    {
        LaunchScope ls(g, KID_NET_RC);
        k_net_rc<R><<<nsb + t.n_big, kRcThreads, 0, g->stream>>>(t, s, x, y, T, (R)g->r, (R)g->c,
                                                                 (R)g->d0, nsb);
    }
    TDP_LAUNCH_CHECK();
    if (g->list_L > 0 && !s.blist) TDP_TRY(dalloc(g, &s.blist, (size_t)t.n_nets * (kMaxK - 1)));
    TDP_TRY(sweep<R>(g));
    return TDP_OK;
}

template tdp_status propagate_impl<float>(tdp_graph *, const float *, const float *, double);
template tdp_status propagate_impl<double>(tdp_graph *, const double *, const double *, double);

template <typename R>
__global__ void k_acc_to_real(const typename Acc<R>::T *a, R *out, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = Acc<R>::val(a[i]);
}

template <typename R>
static tdp_status get_timing_impl(tdp_graph *g, R *arr, R *req, R *slack) {
    State<R> &s = state<R>(g);
    int n = g->topo.n_pins;
    g->n_launch += (arr ? 1 : 0) + (req ? 1 : 0);
    if (arr) k_acc_to_real<R><<<div_up(n, 256), 256, 0, g->stream>>>(s.arr, arr, n);
    if (req) k_acc_to_real<R><<<div_up(n, 256), 256, 0, g->stream>>>(s.req, req, n);
    TDP_LAUNCH_CHECK();
    if (slack)
        TDP_CUDA(cudaMemcpyAsync(slack, s.slack, sizeof(R) * n, cudaMemcpyDeviceToDevice, g->stream));
    return TDP_OK;
}

template <typename R>
static tdp_status get_net_delays_impl(tdp_graph *g, R *tnet, R *cload, R *dcell) {
    State<R> &s = state<R>(g);
    const Topo &t = g->topo;
    if (tnet)
        TDP_CUDA(cudaMemcpyAsync(tnet, s.tnet, sizeof(R) * t.n_pins, cudaMemcpyDeviceToDevice, g->stream));
    if (cload)
        TDP_CUDA(cudaMemcpyAsync(cload, s.cload, sizeof(R) * t.n_nets, cudaMemcpyDeviceToDevice, g->stream));
    if (dcell)
        TDP_CUDA(cudaMemcpyAsync(dcell, s.dnet, sizeof(R) * t.n_nets, cudaMemcpyDeviceToDevice, g->stream));
    return TDP_OK;
}

}  // namespace tdp

using namespace tdp;

extern "C" tdp_status sta_propagate(tdp_graph *g, const void *x_dev, const void *y_dev,
                                    double clock_period_ps, double *wns_out, double *tns_out) {
    if (!g || !x_dev || !y_dev || !std::isfinite(clock_period_ps)) {
        set_error("sta_propagate: NULL graph or positions, or non-finite clock period");
        return TDP_ERR_INVALID;
    }
    tdp_status st = g->prec == TDP_FP32
                        ? propagate_impl<float>(g, (const float *)x_dev, (const float *)y_dev, clock_period_ps)
                        : propagate_impl<double>(g, (const double *)x_dev, (const double *)y_dev, clock_period_ps);
    if (st != TDP_OK) return st;
    g->propagated = true;
    g->extracted = false;
    g->lists_valid_L = g->list_L;
    if (wns_out || tns_out) {
        double h[2];
        const double *src = g->prec == TDP_FP32 ? g->s32.wns_tns : g->s64.wns_tns;
        TDP_CUDA(cudaMemcpyAsync(h, src, sizeof(h), cudaMemcpyDeviceToHost, g->stream));
        TDP_CUDA(cudaStreamSynchronize(g->stream));
        if (wns_out) *wns_out = h[0];
        if (tns_out) *tns_out = h[1];
    }
    return TDP_OK;
}

extern "C" tdp_status sta_get_timing(tdp_graph *g, void *arr_dev, void *req_dev, void *slack_dev) {
    if (!g) {
        set_error("sta_get_timing: NULL graph");
        return TDP_ERR_INVALID;
    }
    if (!g->propagated) {
        set_error("sta_get_timing: call sta_propagate first");
        return TDP_ERR_STATE;
    }
    return g->prec == TDP_FP32
               ? get_timing_impl<float>(g, (float *)arr_dev, (float *)req_dev, (float *)slack_dev)
               : get_timing_impl<double>(g, (double *)arr_dev, (double *)req_dev, (double *)slack_dev);
}

extern "C" tdp_status sta_get_net_delays(tdp_graph *g, void *tnet_dev, void *cload_dev,
                                         void *dcell_dev) {
    if (!g) {
        set_error("sta_get_net_delays: NULL graph");
        return TDP_ERR_INVALID;
    }
    if (!g->propagated) {
        set_error("sta_get_net_delays: call sta_propagate first");
        return TDP_ERR_STATE;
    }
    return g->prec == TDP_FP32
               ? get_net_delays_impl<float>(g, (float *)tnet_dev, (float *)cload_dev, (float *)dcell_dev)
               : get_net_delays_impl<double>(g, (double *)tnet_dev, (double *)cload_dev, (double *)dcell_dev);
}
