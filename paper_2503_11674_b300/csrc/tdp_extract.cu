// report_timing_endpoint(n, K) on the device (Section III-B).
//
// 1. k_viol_collect / k_tile_sort / k_merge_pass / k_sort_finish
//      failing endpoints sorted by (slack, pin): the pin breaks every tie, so
//      the (slack, pin) items are unique and the sorted order is unique.
// 2. sidetrack lists (built by the forward sweep, tdp_sta.cu)
//      For every combinational output v, the cheapest sidetracks on the
//      worst-input chain from v back to its startpoint.  A sidetrack enters a
//      node u through an input pin i other than u's worst input; its cost
//      delta = Arr(worst input) - Arr(i) >= 0 is the slack a path loses by
//      taking it.  list(v) = merge(own sidetracks of v, list(worst-input
//      driver of v)).  Equal costs are ordered as the pin sequences of the
//      resulting paths would be (read from the endpoint).  The forward sweep
//      builds lists as long as the last extraction needed (K - 1); when an
//      extraction needs longer lists it reruns the forward sweep first.
// 3. k_topk: a group of lanes per failing endpoint.  The worst path follows worst
//      inputs from the endpoint; every other path is its parent path plus one
//      sidetrack taken on the parent's last worst-input chain.  A candidate
//      (parent p, index j) is entry j of the list at the head of p's chain;
//      popping it makes a new path and pushes at most two candidates: (p, j+1)
//      and (new path, 0).  Costs only grow along these links, so popping the
//      cheapest candidate K-1 times yields the K lowest-slack paths in order;
//      the frontier never holds more than K candidates, one per lane.
#include <climits>

#include "tdp_internal.cuh"

namespace tdp {

__device__ __forceinline__ bool item_less(const SortItem &a, const SortItem &b) {
    return a.key < b.key || (a.key == b.key && a.pin < b.pin);
}

__device__ __forceinline__ unsigned long long ordered_bits(double v) {
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

template <typename R>
__global__ void k_viol_collect(Topo t, State<R> s, SortItem *items) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool v = false;
    int p = -1;
    double sl = 0.0;
    if (i < t.n_ep) {
        p = t.ep[i];
        sl = (double)s.slack[p];
        v = sl < 0.0;
    }
    unsigned m = __ballot_sync(0xffffffffu, v);
    if (!m) return;
    int lane = threadIdx.x & 31;
    int leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(s.nviol, __popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (v) {
        int off = __popc(m & ((1u << lane) - 1u));
        items[base + off] = SortItem{ordered_bits(sl), (unsigned long long)p};
    }
}

constexpr int kTile = 2048;

// Bitonic sort of one tile of 2048 items in shared memory (1024 threads).
__global__ void __launch_bounds__(1024) k_tile_sort(SortItem *items, const int *nviol) {
    __shared__ SortItem sh[kTile];
    const int n = *nviol;
    const int base = blockIdx.x * kTile;
    if (base >= n) return;
    for (int k = threadIdx.x; k < kTile; k += blockDim.x) {
        int i = base + k;
        sh[k] = i < n ? items[i] : SortItem{~0ull, ~0ull};
    }
    __syncthreads();
    for (int k = 2; k <= kTile; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < kTile; i += blockDim.x) {
                int ixj = i ^ j;
                if (ixj > i) {
                    bool up = (i & k) == 0;
                    SortItem a = sh[i], b = sh[ixj];
                    if (item_less(b, a) == up) {
                        sh[i] = b;
                        sh[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int k = threadIdx.x; k < kTile; k += blockDim.x) {
        int i = base + k;
        if (i < n) items[i] = sh[k];
    }
}

// One merge pass: runs of length `run` are merged pairwise.  Items are
// unique, so an item's output position is its index in its own run plus the
// number of smaller items in the partner run.
__global__ void k_merge_pass(const SortItem *in, SortItem *out, const int *nviol, int run) {
    const int n = *nviol;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const SortItem me = in[i];
    const int r = i / run;
    const int pbeg = (r ^ 1) * run;
    const int pend = min(pbeg + run, n);
    const int pair_base = (r & ~1) * run;
    int cnt = 0;
    if (pbeg < n) {
        int lo = pbeg, hi = pend;
        while (lo < hi) {
            int mid = (lo + hi) >> 1;
            if (item_less(in[mid], me)) lo = mid + 1;
            else hi = mid;
        }
        cnt = lo - pbeg;
    }
    out[pair_base + (i - r * run) + cnt] = me;
}

template <typename R>
__global__ void k_sort_finish(State<R> s, const SortItem *items) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < *s.nviol) s.viol[i] = (int)items[i].pin;
}

// sort items of the failing endpoints listed by pin
template <typename R>
__global__ void k_viol_items(State<R> s, SortItem *items) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < *s.nviol) {
        const int p = s.viol[i];
        items[i] = SortItem{ordered_bits((double)s.slack[p]), (unsigned long long)p};
    }
}

// record k of the sorted order from record i of the pin order (viol ascending)
template <typename R>
__global__ void k_permute_records(State<R> s, const SortItem *sorted, int K, int32_t *viol, int32_t *cnt,
                                  int32_t *par, int32_t *side, int32_t *len, R *cost) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = *s.nviol;
    if (k >= n) return;
    const int pin = (int)sorted[k].pin;
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (s.viol[mid] < pin) lo = mid + 1;
        else hi = mid;
    }
    const int i = lo;
    viol[k] = pin;
    cnt[k] = s.p_count[i];
    for (int r = 0; r < K; ++r) {
        par[(size_t)k * K + r] = s.p_parent[(size_t)i * K + r];
        side[(size_t)k * K + r] = s.p_side[(size_t)i * K + r];
        len[(size_t)k * K + r] = s.p_len[(size_t)i * K + r];
        cost[(size_t)k * K + r] = s.p_cost[(size_t)i * K + r];
    }
}

// Is candidate a (parent path pa + sidetrack pin sa) ordered before candidate
// b (pb + sb) when both have the same slack?  Paths are compared by their pin
// sequences read from the endpoint; two paths first differ at the first
// sidetrack where they disagree, on a shared worst-input chain.
template <typename R>
__device__ bool cand_before(const Topo &t, const State<R> &s, const int *par, const int *side,
                            int pa, int sa, int pb, int sb) {
    int A[kMaxK], B[kMaxK];
    int na = 0, nb = 0;
    A[na++] = sa;
    for (int q = pa; q > 0; q = par[q]) A[na++] = side[q];
    B[nb++] = sb;
    for (int q = pb; q > 0; q = par[q]) B[nb++] = side[q];
    // A[na-1] .. A[0] is the sequence from the endpoint
    for (int k = 0;; ++k) {
        const bool ea = k >= na, eb = k >= nb;
        if (ea && eb) return false;
        if (ea) {
            const int x = B[nb - 1 - k];
            return s.pred[t.sink_onet[x]].x < x;
        }
        if (eb) {
            const int x = A[na - 1 - k];
            return x < s.pred[t.sink_onet[x]].x;
        }
        const int x = A[na - 1 - k], y = B[nb - 1 - k];
        if (x == y) continue;
        const int vx = t.sink_onet[x], vy = t.sink_onet[y];
        if (vx == vy) return x < y;
        if (t.net_level[vx] > t.net_level[vy]) return x < s.pred[vx].x;
        return s.pred[vy].x < y;
    }
}

constexpr int kTopkWarps = 4;

// A warp takes 32 / KP failing endpoints (KP: K rounded up to a power of
// two); the group of KP lanes g * KP .. g * KP + KP - 1 searches endpoint g,
// its frontier one candidate per lane, its paths in shared slots g * KP + r.
// Reductions, ballots and the tie order stay within a group; the warp loops
// until every group is done.
// (at most 32 registers a thread, as the pair walk: four blocks beside a
// block of the backward sweep)
template <typename R>
__global__ void __launch_bounds__(kTopkWarps * 32, 16) k_topk(Topo t, State<R> s, int K, int KP, int G,
                                                          int keep_nonneg, int n_cap) {
    __shared__ int sh_par[kTopkWarps][32], sh_side[kTopkWarps][32];
    __shared__ int sh_len[kTopkWarps][32];
    __shared__ R sh_cost[kTopkWarps][32];
    __shared__ int ct_par[kTopkWarps][32], ct_side[kTopkWarps][32];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int per = 32 / KP, g = lane / KP, gl = lane % KP, gb = g * KP;
    const unsigned gmask = (KP == 32 ? FULL : ((1u << KP) - 1u)) << gb;
    const R INF = (R)__longlong_as_double(0x7ff0000000000000ll);
    chain_enter();
    const int nv = min(*s.nviol, n_cap);
    const int n_tasks = (nv + per - 1) / per;
    for (int task = blockIdx.x * kTopkWarps + w; task < n_tasks; task += gridDim.x * kTopkWarps) {
        const int i = task * per + g;
        const bool have = i < nv;
        const int ep = have ? s.viol[i] : 0;
        const R se = have ? s.slack[ep] : R(0);
        const int e0 = have ? t.pin_net[ep] : 0;
        if (gl == 0 && have) {
            sh_par[w][gb] = -1;
            sh_side[w][gb] = -1;
            sh_len[w][gb] = 1 + s.plen[e0];
            sh_cost[w][gb] = R(0);
        }
        bool cv = false;
        int cpar = 0, cj = 0, ctail = 0;
        R ccost = R(0);
        if (gl == 0 && have && K > 1 && s.bcnt[e0] > 0) {
            const R d = s.blist[(size_t)e0 * G].delta;
            if (keep_nonneg || se + d < R(0)) {
                cv = true;
                ctail = e0;
                ccost = d;
            }
        }
        __syncwarp();
        int n = 1;
        bool done = !have;  // the same in every lane of a group
        for (int step = 1; step < K; ++step) {
            R mn = cv ? ccost : INF;
            for (int o = KP / 2; o > 0; o >>= 1) mn = fmin(mn, __shfl_xor_sync(FULL, mn, o));
            if (!(mn < INF)) done = true;
            if (__all_sync(FULL, done)) break;
            const unsigned tied = __ballot_sync(FULL, !done && cv && ccost == mn) & gmask;
            int win = tied ? __ffs(tied) - 1 : lane;
            if (__any_sync(FULL, __popc(tied) > 1)) {  // equal slack: order by pin sequence
                if (cv) {
                    ct_par[w][lane] = cpar;
                    ct_side[w][lane] = s.blist[(size_t)ctail * G + cj].pin;
                }
                __syncwarp();
                int best = win;
                if (gl == 0 && __popc(tied) > 1) {
                    for (int l = win + 1; l < gb + KP; ++l) {
                        if (!((tied >> l) & 1u)) continue;
                        if (cand_before<R>(t, s, &sh_par[w][gb], &sh_side[w][gb], ct_par[w][l], ct_side[w][l],
                                           ct_par[w][best], ct_side[w][best]))
                            best = l;
                    }
                }
                win = __shfl_sync(FULL, best, gb);
                __syncwarp();
            }
            const int wpar = __shfl_sync(FULL, cpar, win);
            const int wj = __shfl_sync(FULL, cj, win);
            const int wtail = __shfl_sync(FULL, ctail, win);
            const R wcost = __shfl_sync(FULL, ccost, win);
            int sp = 0, tn = 0, len = 0;
            if (!done) {
                sp = s.blist[(size_t)wtail * G + wj].pin;
                tn = t.pin_net[sp];
                len = sh_len[w][gb + wpar] - s.plen[t.sink_onet[sp]] + 2 + s.plen[tn];
            }
            if (gl == 0 && !done) {
                sh_par[w][gb + n] = wpar;
                sh_side[w][gb + n] = sp;
                sh_len[w][gb + n] = len;
                sh_cost[w][gb + n] = wcost;
            }
            if (!done && lane == win) {  // replace the popped candidate by its next sibling
                cv = false;
                if (wj + 1 < min(s.bcnt[wtail], K - 1)) {  // lists may be longer than K - 1
                    const R c2 = sh_cost[w][gb + wpar] + s.blist[(size_t)wtail * G + wj + 1].delta;
                    if (keep_nonneg || se + c2 < R(0)) {
                        cv = true;
                        cj = wj + 1;
                        ccost = c2;
                    }
                }
            }
            bool add_child = false;
            R cc = R(0);
            if (!done && n + 1 < K && s.bcnt[tn] > 0) {
                cc = wcost + s.blist[(size_t)tn * G].delta;
                add_child = keep_nonneg || se + cc < R(0);
            }
            const unsigned freem = __ballot_sync(FULL, !cv) & gmask;
            if (add_child && lane == __ffs(freem) - 1) {
                cv = true;
                cpar = n;
                cj = 0;
                ctail = tn;
                ccost = cc;
            }
            if (!done) ++n;
            __syncwarp();
        }
        for (int r = gl; have && r < n; r += KP) {
            const size_t slot = (size_t)i * K + r;
            s.p_parent[slot] = sh_par[w][gb + r];
            s.p_side[slot] = sh_side[w][gb + r];
            s.p_len[slot] = sh_len[w][gb + r];
            s.p_cost[slot] = sh_cost[w][gb + r];
        }
        if (gl == 0 && have) {
            s.p_count[i] = n;
            atomicAdd((unsigned long long *)s.n_paths, (unsigned long long)n);
        }
        __syncwarp();
    }
}

template <typename R>
static tdp_status ensure_path_buffers(tdp_graph *g, int K) {
    State<R> &s = state<R>(g);
    const Topo &t = g->topo;
    // sized for the largest K, each buffer once (a call that failed part way
    // keeps what it got)
    const size_t slots = (size_t)std::max(t.n_ep, 1) * kMaxK;
    if (!s.p_parent) TDP_TRY(dalloc(g, &s.p_parent, slots));
    if (!s.p_side) TDP_TRY(dalloc(g, &s.p_side, slots));
    if (!s.p_len) TDP_TRY(dalloc(g, &s.p_len, slots));
    if (!s.p_cost) TDP_TRY(dalloc(g, &s.p_cost, slots));
    return TDP_OK;
}

// sort the *nviol items of a (at most n) by (key, pin); the result ends in a
void sort_items(SortItem *&a, SortItem *&b, const int *nviol, int n, cudaStream_t st) {
    k_tile_sort<<<div_up(n, kTile), 1024, 0, st>>>(a, nviol);
    for (int run = kTile; run < n; run *= 2) {
        k_merge_pass<<<div_up(n, 256), 256, 0, st>>>(a, b, nviol, run);
        std::swap(a, b);
    }
}

// failing endpoints listed by pin, and their path records: into (slack, pin)
// order
template <typename R>
static tdp_status sort_viol(tdp_graph *g) {
    if (g->viol_sorted) return TDP_OK;
    State<R> &s = state<R>(g);
    const Topo &t = g->topo;
    cudaStream_t st = g->stream;
    const int K = g->K;
    const size_t slots = (size_t)std::max(t.n_ep, 1) * K;
    SortItem *a = reinterpret_cast<SortItem *>(s.sort_a);
    SortItem *b = reinterpret_cast<SortItem *>(s.sort_b);
    int32_t *viol = nullptr, *cnt = nullptr, *par = nullptr, *side = nullptr, *len = nullptr;
    R *cost = nullptr;
    bool ok = dmalloc_async(&viol, sizeof(int32_t) * std::max(t.n_ep, 1), st) == cudaSuccess &&
              dmalloc_async(&cnt, sizeof(int32_t) * std::max(t.n_ep, 1), st) == cudaSuccess &&
              dmalloc_async(&par, sizeof(int32_t) * slots, st) == cudaSuccess &&
              dmalloc_async(&side, sizeof(int32_t) * slots, st) == cudaSuccess &&
              dmalloc_async(&len, sizeof(int32_t) * slots, st) == cudaSuccess &&
              dmalloc_async(&cost, sizeof(R) * slots, st) == cudaSuccess;
    tdp_status rc = TDP_OK;
    if (!ok) {
        set_error("sta_get_paths: temporary allocation failed");
        rc = TDP_ERR_OOM;
    } else {
        g->n_launch += 2;
        k_viol_items<R><<<div_up(t.n_ep, 256), 256, 0, st>>>(s, a);
        sort_items(a, b, s.nviol, t.n_ep, st);
        k_permute_records<R><<<div_up(t.n_ep, 128), 128, 0, st>>>(s, a, K, viol, cnt, par, side, len, cost);
        cudaMemcpyAsync(s.viol, viol, sizeof(int32_t) * t.n_ep, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(s.p_count, cnt, sizeof(int32_t) * t.n_ep, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(s.p_parent, par, sizeof(int32_t) * slots, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(s.p_side, side, sizeof(int32_t) * slots, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(s.p_len, len, sizeof(int32_t) * slots, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(s.p_cost, cost, sizeof(R) * slots, cudaMemcpyDeviceToDevice, st);
        if (cudaGetLastError() != cudaSuccess) {
            set_error("sta_get_paths: sorting the failing endpoints failed");
            rc = TDP_ERR_CUDA;
        } else {
            g->viol_sorted = true;
        }
    }
    for (void *q : {(void *)viol, (void *)cnt, (void *)par, (void *)side, (void *)len, (void *)cost})
        if (q) cudaFreeAsync(q, st);
    return rc;
}

// failing endpoints sorted by (slack, pin) into viol (nviol cleared first)
template <typename R>
tdp_status sort_failing(tdp_graph *g) {
    Topo &t = g->topo;
    State<R> &s = state<R>(g);
    cudaStream_t st = g->stream;
    TDP_CUDA(cudaMemsetAsync(s.nviol, 0, sizeof(int32_t), st));
    if (t.n_ep > 0) {
        SortItem *a = reinterpret_cast<SortItem *>(s.sort_a);
        SortItem *b = reinterpret_cast<SortItem *>(s.sort_b);
        int passes = 0;
        for (int run = kTile; run < t.n_ep; run *= 2) ++passes;
        LaunchScope ls(g, KID_VIOL_SORT, 3 + passes);
        k_viol_collect<R><<<div_up(t.n_ep, 256), 256, 0, st>>>(t, s, a);
        sort_items(a, b, s.nviol, t.n_ep, st);
        k_sort_finish<R><<<div_up(t.n_ep, 256), 256, 0, st>>>(s, a);
    }
    g->viol_sorted = true;
    TDP_LAUNCH_CHECK();
    return TDP_OK;
}

template tdp_status sort_failing<float>(tdp_graph *);
template tdp_status sort_failing<double>(tdp_graph *);

template <typename R>
tdp_status extract_impl(tdp_graph *g, int n_endpoints, int K, int keep_nonneg) {
    Topo &t = g->topo;
    State<R> &s = state<R>(g);
    cudaStream_t st = g->stream;
    TDP_TRY(ensure_path_buffers<R>(g, K));
    // 1. failing endpoints sorted by (slack, pin)
    if (t.n_ep > 0 && n_endpoints < 0) {
        // all failing endpoints: their order does not change the paths, so
        // they are listed by pin here and sorted when the paths are read; the
        // flags are k_ep_wns's (written with the endpoint slacks), and the
        // compaction writes the count and zeroes the path count
        LaunchScope ls(g, KID_VIOL_SORT, 1);
        TDP_TRY(compact_flags(g, CmpPart{s.ep_flag, t.ep, s.viol, s.nviol, t.n_ep, 1}, nullptr, nullptr,
                              s.n_paths));
        g->viol_sorted = false;
    } else {
        TDP_CUDA(cudaMemsetAsync(s.nviol, 0, sizeof(int32_t), st));
        TDP_CUDA(cudaMemsetAsync(s.n_paths, 0, sizeof(long long), st));
        if (t.n_ep > 0) TDP_TRY(sort_failing<R>(g));
    }
    TDP_LAUNCH_CHECK();
    // 2. sidetrack lists: the next sweeps build K - 1 entries per node; if the
    //    current lists are shorter, rebuild them now with the forward sweep
    if (K > 1 && t.n_ep > 0) {
        g->list_L = list_bucket(K - 1);
        if (g->lists_valid_L < K - 1) {
            join_side(g);  // the rerun rewrites arrival times the backward sweep reads
            TDP_TRY(forward_lists<R>(g));
            g->lists_valid_L = g->list_L;
        }
    }
    // 3. K paths per endpoint
    if (t.n_ep > 0) {
        int n_cap = n_endpoints < 0 ? INT_MAX : n_endpoints;
        int KP = 1;
        while (KP < K) KP *= 2;
        int blocks = std::min(div_up(div_up(t.n_ep, 32 / KP), kTopkWarps), 148 * 16);
        LaunchScope ls(g, KID_TOPK);
        TDP_CUDA(launch_pdl(k_topk<R>, blocks, kTopkWarps * 32, st, t, s, K, KP, list_group(g->lists_valid_L),
                            keep_nonneg, n_cap));
    }
    return TDP_OK;
}

template tdp_status extract_impl<float>(tdp_graph *, int, int, int);
template tdp_status extract_impl<double>(tdp_graph *, int, int, int);

// ---------------------------------------------------------- materialise ---

template <typename R>
__global__ void k_path_lens(State<R> s, int K, int n_use, const int64_t *base, int32_t *lens) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_use) return;
    int c = s.p_count[i];
    for (int r = 0; r < c; ++r) lens[base[i] + r] = s.p_len[(size_t)i * K + r];
}

template <typename R>
__global__ void k_materialise(Topo t, State<R> s, int K, int n_use, const int64_t *base,
                              const int64_t *pin_off, int32_t *ep_out, R *slack_out,
                              int64_t *pin_ptr_out, int32_t *pins_out, int64_t n_paths) {
    int slot = blockIdx.x * blockDim.x + threadIdx.x;
    int i = slot / K, r = slot % K;
    if (i >= n_use || r >= s.p_count[i]) return;
    const int64_t q = base[i] + r;
    const int ep = s.viol[i];
    const size_t sl = (size_t)i * K + r;
    if (ep_out) ep_out[q] = ep;
    if (slack_out) slack_out[q] = s.slack[ep] + s.p_cost[sl];
    if (pin_ptr_out) {
        pin_ptr_out[q] = pin_off[q];
        if (q == n_paths - 1) pin_ptr_out[n_paths] = pin_off[n_paths];
    }
    if (pins_out) {
        int sides[kMaxK];
        int ns = 0;
        for (int x = r; x > 0; x = s.p_parent[(size_t)i * K + x]) sides[ns++] = s.p_side[(size_t)i * K + x];
        const int64_t lo = pin_off[q];
        int64_t pos = lo + s.p_len[sl] - 1;  // written backwards: startpoint first
        walk_path<R>(t, s, ep, sides, ns, [&](int pin, bool) {
            if (pos >= lo) pins_out[pos] = pin;  // never outside this path's range
            --pos;
        });
    }
}

template <typename R>
tdp_status get_paths_impl(tdp_graph *g, int32_t *viol, int32_t *ep, R *slack, int64_t *pin_ptr,
                          int32_t *pins) {
    State<R> &s = state<R>(g);
    const Topo &t = g->topo;
    cudaStream_t st = g->stream;
    if (g->rt_mode) {
        if (viol) {
            int nv = 0;
            TDP_CUDA(cudaMemcpyAsync(&nv, s.nviol, sizeof(int), cudaMemcpyDeviceToHost, st));
            TDP_CUDA(cudaStreamSynchronize(st));
            if (nv > 0) TDP_CUDA(cudaMemcpyAsync(viol, s.viol, sizeof(int32_t) * nv, cudaMemcpyDeviceToDevice, st));
        }
        return rt_get_paths<R>(g, ep, slack, pin_ptr, pins);
    }
    TDP_TRY(sort_viol<R>(g));
    int nv = 0;
    long long np = 0;
    TDP_CUDA(cudaMemcpyAsync(&nv, s.nviol, sizeof(int), cudaMemcpyDeviceToHost, st));
    TDP_CUDA(cudaMemcpyAsync(&np, s.n_paths, sizeof(long long), cudaMemcpyDeviceToHost, st));
    TDP_CUDA(cudaStreamSynchronize(st));
    if (viol && nv > 0)
        TDP_CUDA(cudaMemcpyAsync(viol, s.viol, sizeof(int32_t) * nv, cudaMemcpyDeviceToDevice, st));
    const int n_use = std::min(nv, g->n_endpoints < 0 ? INT_MAX : g->n_endpoints);
    if (np == 0 || n_use == 0 || !(ep || slack || pin_ptr || pins)) {
        if (pin_ptr) TDP_CUDA(cudaMemsetAsync(pin_ptr, 0, sizeof(int64_t), st));
        return TDP_OK;
    }
    int64_t *base = nullptr, *pin_off = nullptr;
    int32_t *lens = nullptr;
    cudaError_t e1 = dmalloc_async(&base, sizeof(int64_t) * (n_use + 1), st);
    cudaError_t e2 = dmalloc_async(&pin_off, sizeof(int64_t) * (np + 1), st);
    cudaError_t e3 = dmalloc_async(&lens, sizeof(int32_t) * np, st);
    tdp_status rc = TDP_OK;
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
        set_error("sta_get_paths: temporary allocation failed");
        rc = TDP_ERR_OOM;
    }
    if (rc == TDP_OK) rc = scan_i32_to_i64(g, s.p_count, base, n_use, st);
    if (rc == TDP_OK) {
        g->n_launch += 2;
        k_path_lens<R><<<div_up(n_use, 256), 256, 0, st>>>(s, g->K, n_use, base, lens);
        rc = scan_i32_to_i64(g, lens, pin_off, np, st);
    }
    if (rc == TDP_OK) {
        int64_t slots = (int64_t)n_use * g->K;
        k_materialise<R><<<div_up(slots, 128), 128, 0, st>>>(t, s, g->K, n_use, base, pin_off, ep,
                                                             slack, pin_ptr, pins, np);
        if (cudaGetLastError() != cudaSuccess) {
            set_error("sta_get_paths: kernel launch failed");
            rc = TDP_ERR_CUDA;
        }
    }
    if (base) cudaFreeAsync(base, st);
    if (pin_off) cudaFreeAsync(pin_off, st);
    if (lens) cudaFreeAsync(lens, st);
    return rc;
}

template tdp_status get_paths_impl<float>(tdp_graph *, int32_t *, int32_t *, float *, int64_t *, int32_t *);
template tdp_status get_paths_impl<double>(tdp_graph *, int32_t *, int32_t *, double *, int64_t *, int32_t *);

}  // namespace tdp

using namespace tdp;

extern "C" tdp_status extract_critical_paths(tdp_graph *g, int32_t n_endpoints, int32_t K,
                                             int32_t keep_nonneg, int64_t *n_paths_out) {
    if (!g || K < 1 || K > kMaxK) {
        set_error("extract_critical_paths: NULL graph or K outside 1..%d", kMaxK);
        return TDP_ERR_INVALID;
    }
    if (!g->propagated) {
        set_error("extract_critical_paths: call sta_propagate first");
        return TDP_ERR_STATE;
    }
    keep_nonneg = keep_nonneg ? 1 : 0;
    g->rt_mode = false;
    tdp_status st = g->prec == TDP_FP32 ? extract_impl<float>(g, n_endpoints, K, keep_nonneg)
                                        : extract_impl<double>(g, n_endpoints, K, keep_nonneg);
    if (st != TDP_OK) return st;
    g->K = K;
    g->keep_nonneg = keep_nonneg;
    g->n_endpoints = n_endpoints;
    g->extracted = true;
    if (n_paths_out) {
        long long h = 0;
        const long long *src = g->prec == TDP_FP32 ? g->s32.n_paths : g->s64.n_paths;
        TDP_CUDA(cudaMemcpyAsync(&h, src, sizeof(h), cudaMemcpyDeviceToHost, g->stream));
        TDP_TRY(check_sync_status(g));  // synchronises the stream
        *n_paths_out = h;
    }
    return TDP_OK;
}

template <typename R>
static tdp_status paths_size_impl(tdp_graph *g, int32_t *nv_out, int64_t *np_out, int64_t *npin_out) {
    State<R> &s = state<R>(g);
    cudaStream_t st = g->stream;
    int nv = 0;
    long long np = 0;
    TDP_CUDA(cudaMemcpyAsync(&nv, s.nviol, sizeof(int), cudaMemcpyDeviceToHost, st));
    TDP_CUDA(cudaMemcpyAsync(&np, s.n_paths, sizeof(long long), cudaMemcpyDeviceToHost, st));
    TDP_CUDA(cudaStreamSynchronize(st));
    if (nv_out) *nv_out = nv;
    if (g->rt_mode) {
        if (np_out) *np_out = g->rt_n_out;
        return npin_out ? rt_paths_size<R>(g, npin_out) : TDP_OK;
    }
    if (np_out) *np_out = np;
    if (npin_out) {
        const int n_use = std::min(nv, g->n_endpoints < 0 ? INT_MAX : g->n_endpoints);
        std::vector<int32_t> cnt(n_use), len((size_t)n_use * g->K);
        if (n_use > 0) {
            TDP_CUDA(cudaMemcpy(cnt.data(), s.p_count, sizeof(int32_t) * n_use, cudaMemcpyDeviceToHost));
            TDP_CUDA(cudaMemcpy(len.data(), s.p_len, sizeof(int32_t) * len.size(), cudaMemcpyDeviceToHost));
        }
        int64_t tot = 0;
        for (int i = 0; i < n_use; ++i)
            for (int r = 0; r < cnt[i]; ++r) tot += len[(size_t)i * g->K + r];
        *npin_out = tot;
    }
    return TDP_OK;
}

extern "C" tdp_status sta_get_paths_size(tdp_graph *g, int32_t *n_viol_out, int64_t *n_paths_out,
                                         int64_t *n_path_pins_out) {
    if (!g) {
        set_error("sta_get_paths_size: NULL graph");
        return TDP_ERR_INVALID;
    }
    if (!g->extracted) {
        set_error("sta_get_paths_size: call extract_critical_paths first");
        return TDP_ERR_STATE;
    }
    return g->prec == TDP_FP32 ? paths_size_impl<float>(g, n_viol_out, n_paths_out, n_path_pins_out)
                               : paths_size_impl<double>(g, n_viol_out, n_paths_out, n_path_pins_out);
}

extern "C" tdp_status sta_get_paths(tdp_graph *g, int32_t *viol_dev, int32_t *ep_dev, void *slack_dev,
                                    int64_t *pin_ptr_dev, int32_t *pins_dev) {
    if (!g) {
        set_error("sta_get_paths: NULL graph");
        return TDP_ERR_INVALID;
    }
    if (!g->extracted) {
        set_error("sta_get_paths: call extract_critical_paths first");
        return TDP_ERR_STATE;
    }
    return g->prec == TDP_FP32
               ? get_paths_impl<float>(g, viol_dev, ep_dev, (float *)slack_dev, pin_ptr_dev, pins_dev)
               : get_paths_impl<double>(g, viol_dev, ep_dev, (double *)slack_dev, pin_ptr_dev, pins_dev);
}
