// report_timing(n) on the device: the n lowest-slack start -> end paths of
// the whole design.  It is the global extraction that Section III-B and
// Table I compare report_timing_endpoint(n, k) against, with OpenTimer's
// semantics: the n most critical endpoints, the n worst paths of each, the
// n worst of those n^2 paths.  Since an endpoint's worst path is no better
// than any other path of it, those are the n lowest-slack paths overall.
//
// Paths form a prefix tree.  The root of endpoint e is its worst path (worst
// inputs from e back to a startpoint), cost 0.  A child is its parent plus
// one sidetrack (a cell input other than the worst one) taken on the
// parent's last worst-input chain: the chain from the endpoint for a root,
// from the driver of the sidetrack's net otherwise.  A sidetrack through
// input i of the cell driving net v costs Arr(worst input of v) - Arr(i) >=
// 0, the slack the path gains by taking it.  Every path is one node, and a
// node's slack (endpoint slack + its cost) is never below its parent's.
//
// So the n lowest-slack nodes form a subtree that holds the parent of each
// of its nodes, and once n nodes of slack <= theta are known, no node of
// slack above theta (nor a descendant of one) can be in the answer.  The
// search runs in rounds over a frontier (the nodes kept in the last round):
//   1. k_rt_expand<false>: a thread per frontier node walks the node's chain
//      and counts its children of slack <= theta; the counts are scanned.
//   2. k_rt_expand<true>: the same walk writes those children at the scanned
//      offsets, in chain order, so that node indices are deterministic.
//   3. k_sel_hist / k_sel_step (radix select, 8 bits a pass): theta becomes
//      the n-th lowest slack among the kept nodes and the new children.
//   4. k_rt_scatter: children of slack <= theta are appended to the kept
//      nodes in order; they are the next frontier.
// Round 0 takes the endpoints' worst paths as its children.  The rounds end
// when no child is within theta.  The kept nodes of slack < theta, and those
// at theta up to n in index order, are sorted by (slack, index): the report,
// worst first.  Equal slacks are thus ordered by the expansion order.
#include <algorithm>
#include <climits>

#include "tdp_internal.cuh"

namespace tdp {

using Key = unsigned long long;

// order-preserving bits of a slack as an unsigned integer
__device__ __forceinline__ Key rt_ord(float v) {
    const uint32_t b = __float_as_uint(v);
    return (Key)((b >> 31) ? ~b : (b | 0x80000000u));
}
__device__ __forceinline__ Key rt_ord(double v) {
    const Key b = (Key)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// state of one radix selection: the bound (the largest key a node may have
// to be kept), the digits fixed so far, the rank still to find among keys
// with those digits, and whether the selection was skipped (fewer than n
// keys within the bound: the bound stays)
struct RtSel {
    Key bound, prefix;
    long long k;
    int skip, pad;
};

constexpr int kRtThreads = 256;

template <typename R>
__global__ void k_rt_root_flags(Topo t, State<R> s, const RtSel *sel, int32_t *flag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < t.n_ep) flag[i] = rt_ord(s.slack[t.ep[i]]) <= sel->bound ? 1 : 0;
}

template <typename R>
__global__ void k_rt_root_write(Topo t, State<R> s, const int32_t *flag, const int64_t *off, RtNodes<R> stg) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= t.n_ep || !flag[i]) return;
    const int ep = t.ep[i];
    const int64_t q = off[i];
    stg.par[q] = -1;
    stg.side[q] = -1;
    stg.ep[q] = ep;
    stg.len[q] = 1 + s.plen[t.pin_net[ep]];
    stg.nsd[q] = 0;
    stg.cost[q] = R(0);
    stg.key[q] = rt_ord(s.slack[ep]);
}

// Chain records of this report (one thread per combinational cell; every
// other net keeps the all -1 record set before): the cell's net gets (net of
// its worst input, its first input, its inputs, the worst input pin), and
// each input the cost of a sidetrack through it, Arr(worst input) - Arr(it)
// (the worst input itself: 0, never used).
template <typename R>
__global__ void k_rt_prep(Topo t, State<R> s) {
    using AC = Acc<R>;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= t.n_comb) return;
    const int e = t.lv_onet[k];
    const int2 pr = s.pred[e];
    const int a = t.lv_in_ptr[k], b = t.lv_in_ptr[k + 1];
    s.rt_chain[e] = make_int4(pr.y, a, b - a, pr.x);
    // input arrivals: the driver's arrival plus the Elmore delay, as the
    // forward sweep forms them
    auto in_arr = [&](int j) { return AC::add(s.arr[t.lv_in_drv[j]], s.tnet[t.lv_in_pin[j]]); };
    typename AC::T aw = AC::ninf();
    for (int j = a; j < b; ++j)
        if (t.lv_in_pin[j] == pr.x) aw = in_arr(j);
    for (int j = a; j < b; ++j) {
        const int p = t.lv_in_pin[j];
        s.rt_delta[j] = p == pr.x ? R(0) : AC::diff(aw, in_arr(j));
    }
}

// Children of frontier node lo + f within the bound: count them (WRITE
// false) or write them at off[f] (WRITE true).  The walk follows the node's
// last worst-input chain from its head net back to the startpoint through
// the chain records (one dependent load a cell; the next record is loaded
// while this cell's inputs are visited) and, at each combinational cell on
// it, visits the inputs other than the worst.
// The frontier holds *nf nodes (read on the device; the grid covers an upper
// bound); the count pass gives the threads beyond it a count of 0.
template <typename R, bool WRITE>
__global__ void __launch_bounds__(kRtThreads) k_rt_expand(Topo t, State<R> s, RtNodes<R> acc, int64_t lo,
                                                         int64_t n_grid, const int64_t *nf, const RtSel *sel,
                                                         int32_t *cnt, const int64_t *off, RtNodes<R> stg) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n_grid) return;
    if (f >= *nf) {
        if (!WRITE) cnt[f] = 0;
        return;
    }
    const int64_t x = lo + f;
    const Key bound = sel->bound;
    int c = 0;
    if (acc.key[x] <= bound) {
        const int ep = acc.ep[x];
        const int side = acc.side[x];
        const R cost = acc.cost[x];
        const R se = s.slack[ep];
        const int len = acc.len[x];
        const int nsd = acc.nsd[x] + 1;
        int64_t pos = WRITE ? off[f] : 0;
        const int64_t end = WRITE ? off[f + 1] : 0;  // never past this node's range
        int e = t.pin_net[side < 0 ? ep : side];
        int4 r = ldg(&s.rt_chain[e]);
        while (r.w >= 0) {  // e is driven by a combinational cell
            const int4 rn = ldg(&s.rt_chain[r.x]);
            for (int j = r.y; j < r.y + r.z; ++j) {
                const int p = ldg(&t.lv_in_pin[j]);
                if (p == r.w) continue;
                const R cc = cost + ldg(&s.rt_delta[j]);
                const Key k = rt_ord(se + cc);
                if (k > bound) continue;
                if (WRITE) {
                    if (pos >= end) break;
                    stg.par[pos] = (int32_t)x;
                    stg.side[pos] = p;
                    stg.ep[pos] = ep;
                    stg.len[pos] = len - s.plen[e] + 2 + s.plen[ldg(&t.lv_in_net[j])];
                    stg.nsd[pos] = nsd;
                    stg.cost[pos] = cc;
                    stg.key[pos] = k;
                    ++pos;
                } else {
                    ++c;
                }
            }
            e = r.x;
            r = rn;
        }
    }
    if (!WRITE) cnt[f] = c;
}

__global__ void k_sel_init(RtSel *sel, long long n) {
    sel->prefix = 0;
    sel->k = n;
    sel->skip = 0;
}

// histogram of digit (key >> shift) & 255 over the keys within the bound
// whose higher digits equal the ones fixed so far
__global__ void __launch_bounds__(kRtThreads) k_sel_hist(const Key *k1, int64_t n1, const Key *k2, int64_t n2,
                                                        const RtSel *sel, int shift, unsigned *hist) {
    __shared__ unsigned h[256];
    h[threadIdx.x] = 0u;
    __syncthreads();
    if (sel->skip) return;
    const Key bound = sel->bound, prefix = sel->prefix;
    const Key hm = shift + 8 >= 64 ? 0ull : (~0ull << (shift + 8));
    const int64_t n = n1 + n2;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const Key k = i < n1 ? k1[i] : k2[i - n1];
        if (k <= bound && ((k ^ prefix) & hm) == 0ull) atomicAdd(&h[(k >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], h[threadIdx.x]);
}

// one block of 256 threads: fix the digit at `shift` (the bucket holding
// the k-th key) and clear the histogram for the next pass; the last pass
// (shift 0) makes the selected key the bound
__global__ void __launch_bounds__(256) k_sel_step(RtSel *sel, unsigned *hist, int shift, int first) {
    __shared__ long long sh[8];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const long long v = hist[tid];
    hist[tid] = 0u;
    const int skip = sel->skip;
    const long long k = sel->k;
    long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    long long before = x - v, total = 0;
    for (int j = 0; j < 8; ++j) {
        if (j < w) before += sh[j];
        total += sh[j];
    }
    if (skip) return;
    if (first && total < k) {
        if (tid == 0) sel->skip = 1;
        return;
    }
    if (before < k && before + v >= k) {
        const Key p = sel->prefix | ((Key)tid << shift);
        sel->prefix = p;
        sel->k = k - before;
        if (shift == 0) sel->bound = p;
    }
}

template <typename R>
__global__ void k_rt_flags_le(const Key *key, int64_t n, const RtSel *sel, int32_t *flag) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = key[i] <= sel->bound ? 1 : 0;
}

template <typename R>
__global__ void k_rt_scatter(RtNodes<R> stg, int64_t n, const RtSel *sel, const int64_t *off, RtNodes<R> acc,
                             int64_t base) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || stg.key[i] > sel->bound) return;
    const int64_t q = base + off[i];
    acc.par[q] = stg.par[i];
    acc.side[q] = stg.side[i];
    acc.ep[q] = stg.ep[i];
    acc.len[q] = stg.len[i];
    acc.nsd[q] = stg.nsd[i];
    acc.cost[q] = stg.cost[i];
    acc.key[q] = stg.key[i];
}

__global__ void k_rt_final_flags(const Key *key, int64_t n, const RtSel *sel, int32_t *fl, int32_t *fe) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Key b = sel->bound, k = key[i];
    fl[i] = k < b ? 1 : 0;
    fe[i] = k == b ? 1 : 0;
}

// the report's nodes as (key, index) items: all below the bound, and those
// at the bound in index order up to n in total
__global__ void k_rt_final_items(const Key *key, int64_t n, const RtSel *sel, const int64_t *offl,
                                 const int64_t *offe, long long n_want, SortItem *items, int *n_sel) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const long long c_less = offl[n], c_eq = offe[n];
    const long long take_eq = max(0ll, min(c_eq, n_want - c_less));
    if (i == 0) *n_sel = (int)(c_less + take_eq);
    if (i >= n) return;
    const Key b = sel->bound, k = key[i];
    if (k < b) items[offl[i]] = SortItem{k, (unsigned long long)i};
    else if (k == b && offe[i] < take_eq) items[c_less + offe[i]] = SortItem{k, (unsigned long long)i};
}

template <typename R>
__global__ void k_rt_out(const SortItem *items, const int *n_sel, RtNodes<R> acc, int32_t *out, int32_t *nsd) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= *n_sel) return;
    const int x = (int)items[q].pin;
    out[q] = x;
    nsd[q] = acc.nsd[x];
}

// sidetracks of reported path q, deepest first
template <typename R>
__global__ void k_rt_sides(RtNodes<R> acc, const int32_t *out, int64_t n, const int64_t *side_off, int32_t *sides) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    int64_t k = side_off[q];
    for (int x = out[q]; acc.nsd[x] > 0; x = acc.par[x]) sides[k++] = acc.side[x];
}

template <typename R>
__global__ void k_rt_lens(RtNodes<R> acc, const int32_t *out, int64_t n, int32_t *lens) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) lens[q] = acc.len[out[q]];
}

template <typename R>
__global__ void k_rt_materialise(Topo t, State<R> s, RtNodes<R> acc, const int32_t *out, int64_t n,
                                 const int64_t *side_off, const int32_t *sides, const int64_t *pin_off,
                                 int32_t *ep_out, R *slack_out, int64_t *pin_ptr_out, int32_t *pins_out) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int x = out[q];
    const int ep = acc.ep[x];
    if (ep_out) ep_out[q] = ep;
    if (slack_out) slack_out[q] = s.slack[ep] + acc.cost[x];
    if (pin_ptr_out) {
        pin_ptr_out[q] = pin_off[q];
        if (q == n - 1) pin_ptr_out[n] = pin_off[n];
    }
    if (pins_out) {
        const int64_t lo = pin_off[q];
        int64_t pos = lo + acc.len[x] - 1;  // written backwards: startpoint first
        walk_path<R>(t, s, ep, sides + side_off[q], acc.nsd[x], [&](int pin, bool) {
            if (pos >= lo) pins_out[pos] = pin;  // never outside this path's range
            --pos;
        });
    }
}

// Eq. (w_ij) accumulation over the reported paths: for every sink on a path
// (its net arc from the net's driver is a pin pair), add q = slack / WNS and
// raise the maximum of q, in the same fixed point as the per-endpoint walk.
template <typename R>
__global__ void k_rt_pair_walk(Topo t, State<R> s, RtNodes<R> acc, const int32_t *out, int64_t n,
                               const int64_t *side_off, const int32_t *sides) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double wns = s.wns_tns[0];
    if (q >= n || !(wns < 0.0)) return;
    const int x = out[q];
    const int ep = acc.ep[x];
    const R sigma = s.slack[ep] + acc.cost[x];
    double qv = (double)sigma / wns;
    qv = fmin(fmax(qv, -kQClamp), kQClamp);
    const long long Q = __double2ll_rn(qv * kQScale);
    walk_path<R>(t, s, ep, sides + side_off[q], acc.nsd[x], [&](int pin, bool is_sink) {
        if (!is_sink) return;
        atomicAdd((unsigned long long *)&s.sumq[pin], (unsigned long long)Q);
        atomicMax(&s.maxq[pin], Q);
    });
}

// ------------------------------------------------------------------ host ---

template <typename T>
static cudaError_t rt_alloc(T **p, int64_t n, cudaStream_t st) {
    *p = nullptr;
    const cudaError_t e = dmalloc_async(p, sizeof(T) * (size_t)std::max<int64_t>(n, 1), st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
    }
    return e;
}

// A temporary device buffer that grows on demand (its contents are dropped
// when it grows) and is freed when the object goes away.
template <typename T>
struct Grow {
    cudaStream_t st;
    T *p = nullptr;
    int64_t cap = 0;
    explicit Grow(cudaStream_t s_) : st(s_) {}
    Grow(const Grow &) = delete;
    bool need(int64_t n) {
        if (n <= cap && p) return true;
        const int64_t nc = std::max<int64_t>(std::max<int64_t>(n, 2 * cap), 1024);
        if (p) cudaFreeAsync(p, st);
        p = nullptr;
        cap = 0;
        if (rt_alloc(&p, nc, st) != cudaSuccess) return false;
        cap = nc;
        return true;
    }
    ~Grow() {
        if (p) cudaFreeAsync(p, st);
    }
};

template <typename R>
struct GrowNodes {
    Grow<int32_t> par, side, ep, len, nsd;
    Grow<R> cost;
    Grow<Key> key;
    explicit GrowNodes(cudaStream_t st) : par(st), side(st), ep(st), len(st), nsd(st), cost(st), key(st) {}
    bool need(int64_t n) {
        return par.need(n) && side.need(n) && ep.need(n) && len.need(n) && nsd.need(n) && cost.need(n) &&
               key.need(n);
    }
    RtNodes<R> view() const { return RtNodes<R>{par.p, side.p, ep.p, len.p, nsd.p, cost.p, key.p}; }
};

template <typename R>
static void nodes_free(RtNodes<R> &a, cudaStream_t st) {
    for (void *p : {(void *)a.par, (void *)a.side, (void *)a.ep, (void *)a.len, (void *)a.nsd, (void *)a.cost,
                    (void *)a.key})
        if (p) cudaFreeAsync(p, st);
    a = RtNodes<R>{};
}

// the kept-node store of the state holds at least `need` nodes, its first
// `keep` nodes preserved
template <typename R>
static tdp_status grow_nodes(tdp_graph *g, int64_t need, int64_t keep) {
    State<R> &s = state<R>(g);
    cudaStream_t st = g->stream;
    if (need <= g->rt_cap && s.rt.par) return TDP_OK;
    const int64_t cap = std::max<int64_t>(need, std::max<int64_t>(2 * g->rt_cap, 1 << 16));
    RtNodes<R> nw;
    const bool ok = rt_alloc(&nw.par, cap, st) == cudaSuccess && rt_alloc(&nw.side, cap, st) == cudaSuccess &&
                    rt_alloc(&nw.ep, cap, st) == cudaSuccess && rt_alloc(&nw.len, cap, st) == cudaSuccess &&
                    rt_alloc(&nw.nsd, cap, st) == cudaSuccess && rt_alloc(&nw.cost, cap, st) == cudaSuccess &&
                    rt_alloc(&nw.key, cap, st) == cudaSuccess;
    if (!ok) {
        nodes_free(nw, st);
        set_error("report_timing: allocation of %lld path nodes failed", (long long)cap);
        return TDP_ERR_OOM;
    }
    if (keep > 0) {
        const size_t k = (size_t)keep;
        const cudaMemcpyKind d2d = cudaMemcpyDeviceToDevice;
        const bool copied = cudaMemcpyAsync(nw.par, s.rt.par, sizeof(int32_t) * k, d2d, st) == cudaSuccess &&
                            cudaMemcpyAsync(nw.side, s.rt.side, sizeof(int32_t) * k, d2d, st) == cudaSuccess &&
                            cudaMemcpyAsync(nw.ep, s.rt.ep, sizeof(int32_t) * k, d2d, st) == cudaSuccess &&
                            cudaMemcpyAsync(nw.len, s.rt.len, sizeof(int32_t) * k, d2d, st) == cudaSuccess &&
                            cudaMemcpyAsync(nw.nsd, s.rt.nsd, sizeof(int32_t) * k, d2d, st) == cudaSuccess &&
                            cudaMemcpyAsync(nw.cost, s.rt.cost, sizeof(R) * k, d2d, st) == cudaSuccess &&
                            cudaMemcpyAsync(nw.key, s.rt.key, sizeof(Key) * k, d2d, st) == cudaSuccess;
        if (!copied) {
            cudaGetLastError();
            nodes_free(nw, st);
            set_error("report_timing: copying the path nodes failed");
            return TDP_ERR_CUDA;
        }
    }
    nodes_free(s.rt, st);
    s.rt = nw;
    g->rt_cap = cap;
    return TDP_OK;
}

// a buffer of the state that holds at least `need` elements (contents dropped)
template <typename T>
static tdp_status grow_buf(tdp_graph *g, T *&p, int64_t &cap, int64_t need) {
    if (need <= cap && p) return TDP_OK;
    const int64_t nc = std::max<int64_t>(std::max<int64_t>(need, 2 * cap), 1024);
    if (p) cudaFreeAsync(p, g->stream);
    p = nullptr;
    cap = 0;
    if (rt_alloc(&p, nc, g->stream) != cudaSuccess) {
        set_error("report_timing: allocation of %lld bytes failed", (long long)(nc * sizeof(T)));
        return TDP_ERR_OOM;
    }
    cap = nc;
    return TDP_OK;
}

static tdp_status read_i64(const int64_t *d, cudaStream_t st, int64_t *h) {
    TDP_CUDA(cudaMemcpyAsync(h, d, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    TDP_CUDA(cudaStreamSynchronize(st));
    return TDP_OK;
}

// two device counts with one synchronisation
static tdp_status read_i64x2(const int64_t *d0, const int64_t *d1, cudaStream_t st, int64_t *h0, int64_t *h1) {
    TDP_CUDA(cudaMemcpyAsync(h0, d0, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    TDP_CUDA(cudaMemcpyAsync(h1, d1, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    TDP_CUDA(cudaStreamSynchronize(st));
    return TDP_OK;
}

// theta := the n-th lowest key among k1[0, n1) and k2[0, n2) within the
// current bound (unchanged when there are fewer than n)
static void select_bound(tdp_graph *g, RtSel *sel, unsigned *hist, const Key *k1, int64_t n1, const Key *k2,
                         int64_t n2, int64_t n, int bits) {
    cudaStream_t st = g->stream;
    const int64_t tot = n1 + n2;
    const int blocks = std::max(1, std::min(div_up(std::max<int64_t>(tot, 1), kRtThreads), g->n_sm * 8));
    k_sel_init<<<1, 1, 0, st>>>(sel, (long long)n);
    for (int shift = bits - 8; shift >= 0; shift -= 8) {
        k_sel_hist<<<blocks, kRtThreads, 0, st>>>(k1, n1, k2, n2, sel, shift, hist);
        k_sel_step<<<1, 256, 0, st>>>(sel, hist, shift, shift == bits - 8);
    }
    g->n_launch += 1 + 2 * (bits / 8);
}

#define RT_NEED(buf, n)                                                  \
    do {                                                                 \
        if (!(buf).need(n)) {                                            \
            set_error("report_timing: temporary allocation failed");     \
            return TDP_ERR_OOM;                                          \
        }                                                                \
    } while (0)

template <typename R>
tdp_status report_impl(tdp_graph *g, int64_t n, int keep_nonneg) {
    Topo &t = g->topo;
    State<R> &s = state<R>(g);
    cudaStream_t st = g->stream;
    constexpr int bits = sizeof(R) == 4 ? 32 : 64;
    g->rt_n_out = 0;
    g->rt_n_sides = 0;
    g->rt_rounds = 0;
    g->rt_nodes = 0;
    TDP_TRY(sort_failing<R>(g));
    if (n == 0 || t.n_ep == 0) return TDP_OK;
    if (!s.rt_chain) TDP_TRY(dalloc(g, &s.rt_chain, (size_t)t.n_nets));
    if (!s.rt_delta) TDP_TRY(dalloc(g, &s.rt_delta, (size_t)std::max(t.n_in, 1)));
    TDP_CUDA(cudaMemsetAsync(s.rt_chain, 0xff, sizeof(int4) * (size_t)t.n_nets, st));
    ++g->n_launch;
    if (t.n_comb > 0) k_rt_prep<R><<<div_up(t.n_comb, kRtThreads), kRtThreads, 0, st>>>(t, s);

    Grow<RtSel> sel(st);
    Grow<unsigned> hist(st);
    Grow<int32_t> flag(st), cnt(st);
    Grow<int64_t> off(st), coff(st);
    GrowNodes<R> stg(st);
    RT_NEED(sel, 1);
    RT_NEED(hist, 256);
    TDP_CUDA(cudaMemsetAsync(hist.p, 0, sizeof(unsigned) * 256, st));
    {
        // bound: slack < 0 (keys up to that of -0, minus one), or any finite slack
        RtSel h{};
        if (keep_nonneg) h.bound = sizeof(R) == 4 ? 0xff800000ull : 0xfff0000000000000ull;  // +inf
        else h.bound = sizeof(R) == 4 ? 0x7ffffffeull : 0x7ffffffffffffffeull;
        TDP_CUDA(cudaMemcpyAsync(sel.p, &h, sizeof(h), cudaMemcpyHostToDevice, st));
    }

    // round 0: the endpoints' worst paths within the bound
    int64_t n_stg = 0;
    RT_NEED(flag, t.n_ep);
    RT_NEED(off, t.n_ep + 1);
    {
        LaunchScope ls(g, KID_RT_EXPAND, 2);
        k_rt_root_flags<R><<<div_up(t.n_ep, kRtThreads), kRtThreads, 0, st>>>(t, s, sel.p, flag.p);
        TDP_TRY(scan_i32_to_i64(g, flag.p, off.p, t.n_ep, st));
        TDP_TRY(read_i64(off.p + t.n_ep, st, &n_stg));
        RT_NEED(stg, n_stg);
        k_rt_root_write<R><<<div_up(t.n_ep, kRtThreads), kRtThreads, 0, st>>>(t, s, flag.p, off.p, stg.view());
        TDP_LAUNCH_CHECK();
    }

    int64_t n_acc = 0;
    while (n_stg > 0) {
        // 3-4: the new bound, then the children within it join the kept nodes
        if (n_acc + n_stg > (int64_t)INT_MAX) {
            set_error("report_timing: more than %d path nodes needed", INT_MAX);
            return TDP_ERR_OOM;
        }
        TDP_TRY(grow_nodes<R>(g, n_acc + n_stg, n_acc));
        const RtNodes<R> sv = stg.view();
        select_bound(g, sel.p, hist.p, s.rt.key, n_acc, sv.key, n_stg, n, bits);
        RT_NEED(flag, n_stg);
        RT_NEED(off, n_stg + 1);
        g->n_launch += 2;
        k_rt_flags_le<R><<<div_up(n_stg, kRtThreads), kRtThreads, 0, st>>>(sv.key, n_stg, sel.p, flag.p);
        TDP_TRY(scan_i32_to_i64(g, flag.p, off.p, n_stg, st));
        k_rt_scatter<R><<<div_up(n_stg, kRtThreads), kRtThreads, 0, st>>>(sv, n_stg, sel.p, off.p, s.rt, n_acc);
        // 1-2: count and scan the children within the bound of the new
        // frontier [n_acc, n_acc + kept), kept = off[n_stg] on the device
        // (the grid covers n_stg >= kept); then one host read of both sizes
        const int64_t lo = n_acc;
        const int64_t *kept_dev = off.p + n_stg;
        RT_NEED(cnt, n_stg);
        RT_NEED(coff, n_stg + 1);
        {
            LaunchScope ls(g, KID_RT_EXPAND);
            k_rt_expand<R, false><<<div_up(n_stg, kRtThreads), kRtThreads, 0, st>>>(t, s, s.rt, lo, n_stg, kept_dev,
                                                                                   sel.p, cnt.p, nullptr, sv);
        }
        TDP_TRY(scan_i32_to_i64(g, cnt.p, coff.p, n_stg, st));
        int64_t kept = 0, n_new = 0;
        TDP_TRY(read_i64x2(kept_dev, coff.p + n_stg, st, &kept, &n_new));
        n_acc += kept;
        if (kept == 0) break;
        ++g->rt_rounds;
        if (n_new == 0) break;
        const int64_t n_grid = n_stg;
        RT_NEED(stg, n_new);
        {
            LaunchScope ls(g, KID_RT_EXPAND);
            k_rt_expand<R, true><<<div_up(n_grid, kRtThreads), kRtThreads, 0, st>>>(t, s, s.rt, lo, n_grid, kept_dev,
                                                                                   sel.p, nullptr, coff.p, stg.view());
        }
        TDP_LAUNCH_CHECK();
        n_stg = n_new;
    }
    g->rt_nodes = n_acc;
    if (n_acc == 0) return TDP_OK;

    // the report: kept nodes below the bound, then those at it, sorted
    const int64_t n_items = std::min<int64_t>(n, n_acc);
    Grow<int32_t> fe(st);
    Grow<int64_t> offe(st);
    Grow<SortItem> ia(st), ib(st);
    Grow<int> n_sel(st);
    RT_NEED(flag, n_acc);
    RT_NEED(fe, n_acc);
    RT_NEED(off, n_acc + 1);
    RT_NEED(offe, n_acc + 1);
    RT_NEED(ia, n_items);
    RT_NEED(ib, n_items);
    RT_NEED(n_sel, 1);
    g->n_launch += 2;
    k_rt_final_flags<<<div_up(n_acc, kRtThreads), kRtThreads, 0, st>>>(s.rt.key, n_acc, sel.p, flag.p, fe.p);
    TDP_TRY(scan_i32_to_i64(g, flag.p, off.p, n_acc, st));
    TDP_TRY(scan_i32_to_i64(g, fe.p, offe.p, n_acc, st));
    k_rt_final_items<<<div_up(n_acc, kRtThreads), kRtThreads, 0, st>>>(s.rt.key, n_acc, sel.p, off.p, offe.p,
                                                                       (long long)n, ia.p, n_sel.p);
    int passes = 0;
    for (int run = 2048; run < n_items; run *= 2) ++passes;
    g->n_launch += 1 + passes;
    SortItem *a = ia.p, *b = ib.p;
    sort_items(a, b, n_sel.p, (int)n_items, st);
    int hn = 0;
    TDP_CUDA(cudaMemcpyAsync(&hn, n_sel.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    TDP_CUDA(cudaStreamSynchronize(st));
    TDP_TRY(grow_buf(g, s.rt_out, g->rt_out_cap, hn));
    TDP_TRY(grow_buf(g, s.rt_side_off, g->rt_soff_cap, hn + 1));
    RT_NEED(cnt, hn);
    g->n_launch += 2;
    k_rt_out<R><<<div_up(std::max(hn, 1), kRtThreads), kRtThreads, 0, st>>>(a, n_sel.p, s.rt, s.rt_out, cnt.p);
    TDP_TRY(scan_i32_to_i64(g, cnt.p, s.rt_side_off, hn, st));
    int64_t n_sides = 0;
    TDP_TRY(read_i64(s.rt_side_off + hn, st, &n_sides));
    TDP_TRY(grow_buf(g, s.rt_sides, g->rt_sides_cap, n_sides));
    k_rt_sides<R><<<div_up(std::max(hn, 1), kRtThreads), kRtThreads, 0, st>>>(s.rt, s.rt_out, hn, s.rt_side_off,
                                                                            s.rt_sides);
    TDP_LAUNCH_CHECK();
    g->rt_n_out = hn;
    g->rt_n_sides = n_sides;
    return TDP_OK;
}

template tdp_status report_impl<float>(tdp_graph *, int64_t, int);
template tdp_status report_impl<double>(tdp_graph *, int64_t, int);

template <typename R>
tdp_status rt_paths_size(tdp_graph *g, int64_t *npin_out) {
    State<R> &s = state<R>(g);
    cudaStream_t st = g->stream;
    const int64_t n = g->rt_n_out;
    *npin_out = 0;
    if (n == 0) return TDP_OK;
    Grow<int32_t> lens(st);
    Grow<int64_t> off(st);
    if (!lens.need(n) || !off.need(n + 1)) {
        set_error("sta_get_paths_size: temporary allocation failed");
        return TDP_ERR_OOM;
    }
    ++g->n_launch;
    k_rt_lens<R><<<div_up(n, kRtThreads), kRtThreads, 0, st>>>(s.rt, s.rt_out, n, lens.p);
    TDP_TRY(scan_i32_to_i64(g, lens.p, off.p, n, st));
    return read_i64(off.p + n, st, npin_out);
}

template tdp_status rt_paths_size<float>(tdp_graph *, int64_t *);
template tdp_status rt_paths_size<double>(tdp_graph *, int64_t *);

template <typename R>
tdp_status rt_get_paths(tdp_graph *g, int32_t *ep, R *slack, int64_t *pin_ptr, int32_t *pins) {
    State<R> &s = state<R>(g);
    const Topo &t = g->topo;
    cudaStream_t st = g->stream;
    const int64_t n = g->rt_n_out;
    if (n == 0 || !(ep || slack || pin_ptr || pins)) {
        if (pin_ptr) TDP_CUDA(cudaMemsetAsync(pin_ptr, 0, sizeof(int64_t), st));
        return TDP_OK;
    }
    Grow<int32_t> lens(st);
    Grow<int64_t> pin_off(st);
    if (!lens.need(n) || !pin_off.need(n + 1)) {
        set_error("sta_get_paths: temporary allocation failed");
        return TDP_ERR_OOM;
    }
    g->n_launch += 2;
    k_rt_lens<R><<<div_up(n, kRtThreads), kRtThreads, 0, st>>>(s.rt, s.rt_out, n, lens.p);
    TDP_TRY(scan_i32_to_i64(g, lens.p, pin_off.p, n, st));
    k_rt_materialise<R><<<div_up(n, 128), 128, 0, st>>>(t, s, s.rt, s.rt_out, n, s.rt_side_off, s.rt_sides,
                                                         pin_off.p, ep, slack, pin_ptr, pins);
    TDP_LAUNCH_CHECK();
    return TDP_OK;
}

template tdp_status rt_get_paths<float>(tdp_graph *, int32_t *, float *, int64_t *, int32_t *);
template tdp_status rt_get_paths<double>(tdp_graph *, int32_t *, double *, int64_t *, int32_t *);

template <typename R>
void rt_pair_walk(tdp_graph *g) {
    State<R> &s = state<R>(g);
    const int64_t n = g->rt_n_out;
    if (n == 0) return;
    LaunchScope ls(g, KID_PAIR_WALK);
    k_rt_pair_walk<R><<<div_up(n, 128), 128, 0, g->stream>>>(g->topo, s, s.rt, s.rt_out, n, s.rt_side_off,
                                                             s.rt_sides);
}

template void rt_pair_walk<float>(tdp_graph *);
template void rt_pair_walk<double>(tdp_graph *);

template <typename R>
static void rt_free_state(tdp_graph *g, State<R> &s) {
    nodes_free(s.rt, g->stream);
    for (void *p : {(void *)s.rt_out, (void *)s.rt_side_off, (void *)s.rt_sides})
        if (p) cudaFreeAsync(p, g->stream);
    s.rt_out = nullptr;
    s.rt_side_off = nullptr;
    s.rt_sides = nullptr;
}

void rt_free(tdp_graph *g) {
    rt_free_state(g, g->s32);
    rt_free_state(g, g->s64);
    g->rt_cap = g->rt_out_cap = g->rt_soff_cap = g->rt_sides_cap = 0;
    cudaStreamSynchronize(g->stream);
}

}  // namespace tdp

using namespace tdp;

extern "C" tdp_status report_timing(tdp_graph *g, int32_t n, int32_t keep_nonneg, int64_t *n_paths_out) {
    if (!g || n < 0) {
        set_error("report_timing: NULL graph or n < 0");
        return TDP_ERR_INVALID;
    }
    if (!g->propagated) {
        set_error("report_timing: call sta_propagate first");
        return TDP_ERR_STATE;
    }
    keep_nonneg = keep_nonneg ? 1 : 0;
    g->rt_mode = true;
    g->extracted = false;
    tdp_status st = g->prec == TDP_FP32 ? report_impl<float>(g, n, keep_nonneg)
                                        : report_impl<double>(g, n, keep_nonneg);
    if (st != TDP_OK) {
        g->rt_n_out = 0;
        return st;
    }
    g->keep_nonneg = keep_nonneg;
    g->extracted = true;
    if (n_paths_out) {
        TDP_TRY(check_sync_status(g));
        *n_paths_out = g->rt_n_out;
    }
    return TDP_OK;
}
