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

template <typename R>
__device__ __forceinline__ BEnt<R> bent_none() {
    return BEnt<R>{(R)__longlong_as_double(0x7ff0000000000000ll), -1};
}

// Sidetrack list of one node (Section III-B extraction): the L cheapest
// deviations on the worst-input chain from the node back to its startpoint.
// A deviation enters a node through an input other than its worst one; its
// cost is Arr(worst input) - Arr(that input).  The list is the merge of the
// node's own deviations with the list of its worst input's driver.  Equal
// costs are ordered as the resulting paths' pin sequences (read from the
// endpoint) would be: own deviations through a pin below the worst input,
// then the inherited entries, then own deviations through a pin above it.
// Lists hold exactly L entries; unused ones are +inf sentinels (pin -1).
template <typename R>
__device__ __forceinline__ void build_sidetracks(const Topo &t, State<R> &s, int e, int bi,
                                                 int bn, bool bn_comb,
                                                 typename Acc<R>::T best, const int *ip,
                                                 const typename Acc<R>::T *ain, int nin, int L) {
    using AC = Acc<R>;
    BEnt<R> pl[kMaxK - 1];
    if (bn_comb) {  // issue the inherited list's loads before anything else
        const BEnt<R> *src = s.blist + (size_t)bn * L;
        for (int j = 0; j < L; ++j) pl[j] = ldg(&src[j]);
    }
    R od[kMaxFanin];
    int op[kMaxFanin];
    int no = 0;
    for (int u = 0; u < nin; ++u) {
        const int i = ip[u];
        if (i == bi) continue;
        const R d = AC::diff(best, ain[u]);
        int pos = no;
        while (pos > 0) {  // insertion by (delta, side of the worst input, pin)
            const R dp = od[pos - 1];
            const int pp = op[pos - 1];
            const bool before = d < dp || (d == dp && ((i < bi) != (pp < bi) ? (i < bi) : i < pp));
            if (!before) break;
            od[pos] = dp;
            op[pos] = pp;
            --pos;
        }
        od[pos] = d;
        op[pos] = i;
        ++no;
    }
    BEnt<R> *out = s.blist + (size_t)e * L;
    int ia = 0, ib = 0, m = 0;
    for (; m < L; ++m) {
        const bool ha = ia < no;
        const bool hb = bn_comb && ib < L && pl[ib].pin >= 0;
        if (!ha && !hb) break;
        bool take_own;
        if (!hb) take_own = true;
        else if (!ha) take_own = false;
        else take_own = od[ia] < pl[ib].delta || (od[ia] == pl[ib].delta && op[ia] < bi);
        if (take_own) {
            out[m] = BEnt<R>{od[ia], op[ia]};
            ++ia;
        } else {
            out[m] = pl[ib];
            ++ib;
        }
    }
    s.bcnt[e] = m;
    for (int j = m; j < L; ++j) out[j] = bent_none<R>();
}

template <typename R>
__global__ void __launch_bounds__(kLvThreads) k_fwd_level(Topo t, State<R> s, int lo, int hi, int L) {
    using AC = Acc<R>;
    using A = typename AC::T;
    const int k = lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= hi) return;
    const int a = ldg(&t.lv_in_ptr[k]), b = ldg(&t.lv_in_ptr[k + 1]);
    const int e = ldg(&t.lv_onet[k]), o = ldg(&t.lv_out[k]);
    const R dcell = ldg(&s.dnet[e]);
    // inputs ascending by pin: strict > keeps the lowest pin on ties (and the
    // first input if arrivals are not comparable)
    int bi = -1, bn = -1, bl = 0;
    bool bc = false;
    A best = AC::ninf();
    int ipa[kMaxFanin];
    A ain[kMaxFanin];
    for (int q0 = a; q0 < b; q0 += kPre) {
        int ip[kPre], in[kPre], dv[kPre], pl[kPre];
        uint8_t cb[kPre];
        A av[kPre];
        R tv[kPre];
#pragma unroll
        for (int u = 0; u < kPre; ++u) {
            if (q0 + u < b) {
                ip[u] = ldg(&t.lv_in_pin[q0 + u]);
                in[u] = ldg(&t.lv_in_net[q0 + u]);
                dv[u] = ldg(&t.lv_in_drv[q0 + u]);
                cb[u] = ldg(&t.lv_in_comb[q0 + u]);
            }
        }
#pragma unroll
        for (int u = 0; u < kPre; ++u) {
            if (q0 + u < b) {
                av[u] = ldg(&s.arr[dv[u]]);
                tv[u] = ldg(&s.tnet[ip[u]]);
                pl[u] = ldg(&s.plen[in[u]]);
            }
        }
#pragma unroll
        for (int u = 0; u < kPre; ++u) {
            if (q0 + u < b) {
                const A v = AC::add(av[u], tv[u]);
                s.arr[ip[u]] = v;
                ipa[q0 - a + u] = ip[u];
                ain[q0 - a + u] = v;
                if (bi < 0 || AC::gt(v, best)) {
                    best = v;
                    bi = ip[u];
                    bn = in[u];
                    bl = pl[u];
                    bc = cb[u];
                }
            }
        }
    }
    s.arr[o] = AC::add(best, dcell);
    s.pred_in[e] = bi;
    s.pred_net[e] = bn;
    s.plen[e] = bl + 2;
    if (L > 0) build_sidetracks<R>(t, s, e, bi, bn, bc, best, ipa, ain, b - a, L);
}

// ----------------------------------------------------------- backward ---

// req / slack of the sinks first, first+step, ... < b of a net whose driver
// has arrival ad; returns min over them of req(s) - t(s).
template <typename R>
__device__ __forceinline__ typename Acc<R>::T net_sinks_req(const Topo &t, State<R> &s, int first,
                                                            int b, int step,
                                                            typename Acc<R>::T ad,
                                                            typename Acc<R>::T Tacc) {
    using AC = Acc<R>;
    using A = typename AC::T;
    A m = AC::pinf();
    for (int p0 = first; p0 < b; p0 += kPre * step) {
        uint8_t kd[kPre];
        R tp[kPre];
        int so[kPre], sn[kPre];
#pragma unroll
        for (int u = 0; u < kPre; ++u) {
            const int p = p0 + u * step;
            if (p < b) {
                kd[u] = ldg(&t.pin_kind[p]);
                tp[u] = ldg(&s.tnet[p]);
                so[u] = ldg(&t.sink_out[p]);
                sn[u] = ldg(&t.sink_onet[p]);
            }
        }
        A rq[kPre], ap[kPre];
#pragma unroll
        for (int u = 0; u < kPre; ++u) {
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
        for (int u = 0; u < kPre; ++u) {
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

// One warp per task of this level (tasks [lo, hi) of the backward list).
template <typename R>
__global__ void __launch_bounds__(kLvThreads) k_bwd_level(Topo t, State<R> s, int lo, int hi) {
    using AC = Acc<R>;
    using A = typename AC::T;
    const int w = lo + (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (w >= hi) return;
    const A Tacc = acc_from_double<R>(*s.T);
    const BwTask task = t.bw_task[w];
    if (task.kind == 0) {
        if (lane >= task.p1) return;
        const int e = ldg(&t.bw_nets[task.p0 + lane]);
        const int a = ldg(&t.net_ptr[e]), b = ldg(&t.net_ptr[e + 1]);
        const A ad = ldg(&s.arr[a]);
        const A m = net_sinks_req<R>(t, s, a + 1, b, 1, ad, Tacc);
        s.req[a] = m;
        s.slack[a] = AC::diff(m, ad);
        return;
    }
    const int a = ldg(&t.net_ptr[task.net]);
    const A ad = ldg(&s.arr[a]);
    A m = net_sinks_req<R>(t, s, task.p0 + lane, task.p1, 32, ad, Tacc);
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
            k_fwd_level<R><<<div_up(hi - lo, kLvThreads), kLvThreads, 0, cs>>>(t, s, lo, hi, L);
            ++nk;
        }
        ok = cudaGetLastError() == cudaSuccess;
    }
    for (int l = t.depth; bwd && l >= 0 && ok; --l) {
        const int lo = g->lv.bw_lo[l], hi = g->lv.bw_hi[l];
        if (hi > lo) {
            k_bwd_level<R><<<div_up((int64_t)(hi - lo) * 32, kLvThreads), kLvThreads, 0, cs>>>(t, s, lo, hi);
            ++nk;
        }
        ok = cudaGetLastError() == cudaSuccess;
    }
    if (bwd && ok) {
        k_wns_tns<R><<<kRedBlocks, kRedThreads, 0, cs>>>(t, s);
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

// Forward and backward sweeps and WNS / TNS, one graph replay.  The forward
// sweep also builds sidetrack lists of length g->list_L (0: none).
template <typename R>
static tdp_status sweep(tdp_graph *g) {
    if (!g->sta_graph || g->sta_graph_L != g->list_L) {
        if (g->sta_graph) cudaGraphExecDestroy(g->sta_graph);
        g->sta_graph = nullptr;
        TDP_TRY(capture<R>(g, &g->sta_graph, &g->sta_graph_kernels, true, true, g->list_L));
        g->sta_graph_L = g->list_L;
    }
    g->n_launch += g->sta_graph_kernels;
    TDP_CUDA(cudaGraphLaunch(g->sta_graph, g->stream));
    return TDP_OK;
}

// Forward sweep only, rebuilding sidetrack lists of length g->list_L.  The
// arrival times it writes are identical to the ones already there.
template <typename R>
tdp_status forward_lists(tdp_graph *g) {
    State<R> &s = state<R>(g);
    if (!s.blist) TDP_TRY(dalloc(g, &s.blist, (size_t)g->topo.n_nets * (kMaxK - 1)));
    if (!g->fwd_graph || g->fwd_graph_L != g->list_L) {
        if (g->fwd_graph) cudaGraphExecDestroy(g->fwd_graph);
        g->fwd_graph = nullptr;
        TDP_TRY(capture<R>(g, &g->fwd_graph, &g->fwd_graph_kernels, true, false, g->list_L));
        g->fwd_graph_L = g->list_L;
    }
    g->n_launch += g->fwd_graph_kernels;
    TDP_CUDA(cudaGraphLaunch(g->fwd_graph, g->stream));
    return TDP_OK;
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
