// Static timing analysis on the device (Section II-B; Eq. (2) slack;
// Eqs. (3)-(4) WNS/TNS; Eq. (8) Elmore net delay).
//
//   k_net_rc     one pass over the nets: pin positions, Elmore delay of every
//                sink, net load and driving-cell delay (thread per net up to 32
//                sinks, warp per net above, FP64 load sum there)
//   k_fwd_level  arrival times of the combinational cells of one level
//                (thread per cell; max / argmax over its inputs)
//   k_bwd_level  required times of the nets driven from one level
//                (thread per net, warp per high-fanout net; min over sinks)
//   k_wns_tns    FP64 WNS / TNS over the endpoints (fixed-order reduction)
//
// The per-level launches are captured once into a CUDA graph and replayed.
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

template <typename R>
__device__ __forceinline__ void net_finish(const Topo &t, State<R> &s, int e, int drv, int cd,
                                           double load, R d0) {
    R ld = (R)load;
    s.cload[e] = ld;
    R dd = d0 + s.cell_rdrv[cd] * ld;
    s.dnet[e] = dd;
    if (t.pin_kind[drv] == PK_START) s.arr[drv] = Acc<R>::make(dd);
}

template <typename R>
__global__ void __launch_bounds__(256) k_net_rc(Topo t, State<R> s, const R *__restrict__ x,
                                                const R *__restrict__ y, double T, R r, R c, R d0,
                                                int n_small_warps) {
    const int gw = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (blockIdx.x == 0 && threadIdx.x == 0) *s.T = T;
    if (gw < n_small_warps) {
        int e = gw * 32 + lane;
        if (e >= t.n_nets) return;
        int a = t.net_ptr[e], b = t.net_ptr[e + 1];
        if (b - a - 1 > kBigFanout) return;
        int cd = t.pin_cell[a];
        R xd = x[cd] + s.pin_dx[a], yd = y[cd] + s.pin_dy[a];
        R load = 0;
        for (int p = a + 1; p < b; ++p) {
            int cs = t.pin_cell[p];
            R L = fabs(x[cs] + s.pin_dx[p] - xd) + fabs(y[cs] + s.pin_dy[p] - yd);
            R Rw = r * L, Cw = c * L;
            R cap = s.pin_cap[p];
            s.tnet[p] = Rw * (Cw * R(0.5) + cap);
            load += Cw + cap;
        }
        net_finish(t, s, e, a, cd, (double)load, d0);
    } else {
        int k = gw - n_small_warps;
        if (k >= t.n_big) return;
        int e = t.big_nets[k];
        int a = t.net_ptr[e], b = t.net_ptr[e + 1];
        int cd = t.pin_cell[a];
        R xd = x[cd] + s.pin_dx[a], yd = y[cd] + s.pin_dy[a];
        double load = 0.0;
        for (int p = a + 1 + lane; p < b; p += 32) {
            int cs = t.pin_cell[p];
            R L = fabs(x[cs] + s.pin_dx[p] - xd) + fabs(y[cs] + s.pin_dy[p] - yd);
            R Rw = r * L, Cw = c * L;
            R cap = s.pin_cap[p];
            s.tnet[p] = Rw * (Cw * R(0.5) + cap);
            load += (double)(Cw + cap);
        }
        for (int o = 16; o > 0; o >>= 1) load += __shfl_xor_sync(0xffffffffu, load, o);
        if (lane == 0) net_finish(t, s, e, a, cd, load, d0);
    }
}

template <typename R>
__global__ void __launch_bounds__(128) k_fwd_level(Topo t, State<R> s, int lo, int hi) {
    using AC = Acc<R>;
    using A = typename AC::T;
    const int k = lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= hi) return;
    const int a = t.lv_in_ptr[k], b = t.lv_in_ptr[k + 1];
    // inputs ascending by pin: strict > keeps the lowest pin on ties (and the
    // first input if arrivals are not comparable)
    int bi = t.lv_in_pin[a], bn = t.lv_in_net[a];
    A best = AC::add(s.arr[t.lv_in_drv[a]], s.tnet[bi]);
    s.arr[bi] = best;
    for (int q = a + 1; q < b; ++q) {
        const int i = t.lv_in_pin[q];
        A v = AC::add(s.arr[t.lv_in_drv[q]], s.tnet[i]);
        s.arr[i] = v;
        if (AC::gt(v, best)) {
            best = v;
            bi = i;
            bn = t.lv_in_net[q];
        }
    }
    const int e = t.lv_onet[k];
    s.arr[t.lv_out[k]] = AC::add(best, s.dnet[e]);
    s.pred_in[e] = bi;
    s.pred_net[e] = bn;
    s.plen[e] = s.plen[bn] + 2;
}

// Required time of one sink and its contribution to the driver's required time.
template <typename R>
__device__ __forceinline__ typename Acc<R>::T sink_req(const Topo &t, State<R> &s, int p,
                                                       typename Acc<R>::T ad,
                                                       typename Acc<R>::T Tacc) {
    using AC = Acc<R>;
    using A = typename AC::T;
    const R tp = s.tnet[p];
    A rq, ap;
    if (t.pin_kind[p] == PK_ENDPOINT) {
        ap = AC::add(ad, tp);
        s.arr[p] = ap;
        rq = Tacc;
    } else {
        rq = AC::add(s.req[t.sink_out[p]], -s.dnet[t.sink_onet[p]]);
        ap = s.arr[p];
    }
    s.req[p] = rq;
    s.slack[p] = AC::diff(rq, ap);
    return AC::add(rq, -tp);
}

template <typename R>
__global__ void __launch_bounds__(128) k_bwd_level(Topo t, State<R> s, int lo, int nsmall, int hi) {
    using AC = Acc<R>;
    using A = typename AC::T;
    const int gw = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    const int nsw = (nsmall + 31) >> 5;
    const A Tacc = acc_from_double<R>(*s.T);
    if (gw < nsw) {
        const int idx = lo + gw * 32 + lane;
        if (idx >= lo + nsmall) return;
        const int e = t.bl_net[idx];
        const int a = t.net_ptr[e], b = t.net_ptr[e + 1];
        const A ad = s.arr[a];
        A m = AC::pinf();
        for (int p = a + 1; p < b; ++p) {
            A cand = sink_req<R>(t, s, p, ad, Tacc);
            if (AC::lt(cand, m)) m = cand;
        }
        s.req[a] = m;
        s.slack[a] = AC::diff(m, ad);
    } else {
        const int idx = lo + nsmall + (gw - nsw);
        if (idx >= hi) return;
        const int e = t.bl_net[idx];
        const int a = t.net_ptr[e], b = t.net_ptr[e + 1];
        const A ad = s.arr[a];
        A m = AC::pinf();
        for (int p = a + 1 + lane; p < b; p += 32) {
            A cand = sink_req<R>(t, s, p, ad, Tacc);
            if (AC::lt(cand, m)) m = cand;
        }
        for (int o = 16; o > 0; o >>= 1) {  // min is exact: the order does not matter
            A other;
            if constexpr (sizeof(A) == 8 && sizeof(R) == 4) {
                other.hi = __shfl_xor_sync(0xffffffffu, m.hi, o);
                other.lo = __shfl_xor_sync(0xffffffffu, m.lo, o);
            } else {
                other = __shfl_xor_sync(0xffffffffu, m, o);
            }
            if (AC::lt(other, m)) m = other;
        }
        if (lane == 0) {
            s.req[a] = m;
            s.slack[a] = AC::diff(m, ad);
        }
    }
}

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

template <typename R>
static tdp_status capture_sta_graph(tdp_graph *g) {
    Topo &t = g->topo;
    State<R> &s = state<R>(g);
    cudaStream_t cs = g->cap_stream;
    TDP_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    bool ok = true;
    for (int l = 1; l <= t.depth && ok; ++l) {
        int lo = g->lv.lvl_ptr[l - 1], hi = g->lv.lvl_ptr[l];
        if (hi > lo) k_fwd_level<R><<<div_up(hi - lo, 128), 128, 0, cs>>>(t, s, lo, hi);
        ok = cudaGetLastError() == cudaSuccess;
    }
    for (int l = t.depth; l >= 0 && ok; --l) {
        int lo = g->lv.bl_ptr[l], hi = g->lv.bl_ptr[l + 1], ns = g->lv.bl_small[l];
        int warps = div_up(ns, 32) + (hi - lo - ns);
        if (warps > 0) k_bwd_level<R><<<div_up((int64_t)warps * 32, 128), 128, 0, cs>>>(t, s, lo, ns, hi);
        ok = cudaGetLastError() == cudaSuccess;
    }
    if (ok) {
        k_wns_tns<R><<<kRedBlocks, kRedThreads, 0, cs>>>(t, s);
        ok = cudaGetLastError() == cudaSuccess;
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &graph);
    if (!ok || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        set_error("sta_propagate: capturing the level sweep failed: %s",
                  cudaGetErrorString(e != cudaSuccess ? e : cudaGetLastError()));
        return TDP_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&g->sta_graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        g->sta_graph = nullptr;
        set_error("sta_propagate: cudaGraphInstantiate failed: %s", cudaGetErrorString(e));
        return TDP_ERR_CUDA;
    }
    return TDP_OK;
}

template <typename R>
tdp_status propagate_impl(tdp_graph *g, const R *x, const R *y, double T) {
    Topo &t = g->topo;
    State<R> &s = state<R>(g);
    int nsw = div_up(t.n_nets, 32);
    int64_t threads = (int64_t)(nsw + t.n_big) * 32;
    k_net_rc<R><<<div_up(threads, 256), 256, 0, g->stream>>>(t, s, x, y, T, (R)g->r, (R)g->c,
                                                             (R)g->d0, nsw);
    TDP_LAUNCH_CHECK();
    if (!g->sta_graph) TDP_TRY(capture_sta_graph<R>(g));
    TDP_CUDA(cudaGraphLaunch(g->sta_graph, g->stream));
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
