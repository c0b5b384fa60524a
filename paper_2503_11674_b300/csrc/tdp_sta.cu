// Static timing analysis on the device (Section II-B; Eq. (2) slack;
// Eqs. (3)-(4) WNS/TNS; Eq. (8) Elmore net delay).
//
//   k_net_rc     one pass over the nets: pin positions, Elmore delay of every
//                sink, net load and driving-cell delay (thread per net up to 32
//                sinks, block per net above, FP64 load sum there)
//   k_fwd_sweep  the forward sweep in one cooperative launch: arrival times
//                level by level (thread per combinational cell: max / argmax
//                over its inputs), and, when asked, each cell's sidetrack list
//                for report_timing_endpoint; grid-wide barrier between levels
//   k_bwd_sweep  the backward sweep in one cooperative launch: required times
//                of the nets driven from each level, deepest first (lane per
//                net of at most 8 sinks, warp per 128 sinks of larger nets,
//                split nets combined by the last warp to finish), then WNS /
//                TNS over the endpoints (FP64, fixed-order reduction)
//
// Where a cooperative launch cannot be made resident (or TDP_LEVEL_GRAPHS=1),
// the same per-cell and per-task code runs as one launch per level
// (k_fwd_level, k_bwd_level, k_wns_tns) captured in CUDA graphs; there every
// array a level reads was written by an earlier launch, so the reads use the
// read-only path.  Inside one cooperative launch, values written before a
// barrier are read from L2.  Either way all loads of a group of inputs /
// sinks are issued before the first store.
#include <algorithm>
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

// Entries compare by cost, then key: a strict total order (costs as
// order-preserving integer bits), so the merge below ranks every entry of a
// list uniquely.
__device__ __forceinline__ uint32_t ord_bits(float d) {
    const uint32_t u = __float_as_uint(d);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ uint64_t ord_bits(double d) {
    const uint64_t u = (uint64_t)__double_as_longlong(d);
    return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}

template <typename R>
__device__ __forceinline__ bool lent_before(const LEnt<R> &a, const LEnt<R> &b) {
    const auto ua = ord_bits(a.d), ub = ord_bits(b.d);
    return ua < ub || (ua == ub && a.key < b.key);
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
// exactly L entries; unused ones are +inf sentinels (pin -1).  A net's list
// starts at entry net * G, G = list_group(L) (one aligned block of G entries).

__device__ __forceinline__ LEnt<float> lent_of(const BEnt<float> &v) {
    return LEnt<float>{v.delta, v.pin < 0 ? kNoneKey : ((1u << 29) | (uint32_t)v.pin)};
}
__device__ __forceinline__ LEnt<double> lent_of(const BEnt<double> &v) {
    return LEnt<double>{v.delta, v.pin < 0 ? kNoneKey : ((1u << 29) | (uint32_t)v.pin)};
}
template <typename R>
__device__ __forceinline__ BEnt<R> bent_of(const LEnt<R> &x) {
    return BEnt<R>{x.d, x.key == kNoneKey ? -1 : (int32_t)(x.key & kPinMask)};
}

// ---- one cell per thread (cells with more inputs than a group has lanes)

// A cell with more inputs than a group has lanes (rare): one thread visits
// its inputs kPre at a time (arrival / argmax), then builds the list in
// place in its output block, inserting the own deviations one by one.
// While it is built, an entry's pin field holds its ordering key.
template <typename R, int L, bool COH>
__device__ __noinline__ void fwd_cell_wide(const Topo &t, State<R> &s, int k, int a, int b) {
    using AC = Acc<R>;
    using A = typename AC::T;
    constexpr int G = list_group(L);
    const int e = ldg(&t.lv_onet[k]), o = ldg(&t.lv_out[k]);
    int bi = -1, bp = a;
    A best = AC::ninf();
    for (int p0 = a; p0 < b; p0 += kPre) {
        int ip[kPre], dv[kPre];
        A av[kPre];
        R tv[kPre];
#pragma unroll
        for (int u = 0; u < kPre; ++u) {
            if (p0 + u < b) {
                ip[u] = ldg(&t.lv_in_pin[p0 + u]);
                dv[u] = ldg(&t.lv_in_drv[p0 + u]);
            }
        }
#pragma unroll
        for (int u = 0; u < kPre; ++u) {
            if (p0 + u < b) {
                av[u] = ldd<COH>(&s.arr[dv[u]]);
                tv[u] = ldg(&s.tnet[ip[u]]);
            }
        }
#pragma unroll
        for (int u = 0; u < kPre; ++u) {
            if (p0 + u < b) {
                av[u] = AC::add(av[u], tv[u]);
                s.arr[ip[u]] = av[u];
                // largest arrival, lowest pin on ties (the group order below)
                if (bi < 0 || AC::gt(av[u], best) || (!AC::gt(best, av[u]) && ip[u] < bi)) {
                    best = av[u];
                    bi = ip[u];
                    bp = p0 + u;
                }
            }
        }
    }
    const int bn = ldg(&t.lv_in_net[bp]);
    const bool bc = (ldg(&t.lv_in_flags[bp]) & kInComb) != 0;
    s.arr[o] = AC::add(best, ldg(&s.dnet[e]));
    s.pred_in[e] = bi;
    s.pred_net[e] = bn;
    s.plen[e] = ldd<COH>(&s.plen[bn]) + 2;
    if constexpr (L > 0) {
        BEnt<R> *out = s.blist + (size_t)e * G;
        const BEnt<R> *src = s.blist + (size_t)bn * G;
        for (int j = 0; j < L; ++j) {
            const LEnt<R> x = bc ? lent_of(ldd<COH>(&src[j])) : LEnt<R>{r_inf<R>(), kNoneKey};
            out[j] = BEnt<R>{x.d, (int32_t)x.key};
        }
        for (int p = a; p < b; ++p) {
            const int ip = ldg(&t.lv_in_pin[p]);
            if (ip == bi) continue;
            const A av = ldcg(&s.arr[ip]);  // stored above by this thread
            const LEnt<R> x{AC::diff(best, av), ((ip < bi ? 0u : 2u) << 29) | (uint32_t)ip};
            int j = 0;
            for (; j < L; ++j) {
                const BEnt<R> y = ldcg(&out[j]);
                if (lent_before(x, LEnt<R>{y.delta, (uint32_t)y.pin})) break;
            }
            if (j == L) continue;
            for (int q = L - 1; q > j; --q) out[q] = ldcg(&out[q - 1]);
            out[j] = BEnt<R>{x.d, (int32_t)x.key};
        }
        int m = 0;
        for (int j = 0; j < L; ++j) {
            BEnt<R> y = ldcg(&out[j]);
            const uint32_t key = (uint32_t)y.pin;
            y.pin = key == kNoneKey ? -1 : (int32_t)(key & kPinMask);
            m += key == kNoneKey ? 0 : 1;
            out[j] = y;
        }
        s.bcnt[e] = m;
    }
}

// ---- one cell per group of G lanes (the common case)

template <typename T>
__device__ __forceinline__ T shfl_idx(T v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ fx2 shfl_idx(fx2 v, int src) {
    return fx2{__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src)};
}
template <typename T>
__device__ __forceinline__ T shfl_x(T v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ fx2 shfl_x(fx2 v, int o) {
    return fx2{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}

// What one lane of a group knows about its group's cell k (k < 0: none) and
// about the input with index gl (the lane's index in the group), if any:
// its pin, net, driver pin and flags, and, once loaded, its Elmore delay
// (has_tv) and its driver's arrival and chain length (has_old).
template <typename R>
struct LaneTopo {
    using A = typename Acc<R>::T;
    int k, a, b, e, o;
    int ip, in, dv, fl;
    bool has_tv, has_old;
    R tv;
    A ad;
    int pl;
};

// Topology of cell k for lane gl.  With old_vals (single launch, before the
// barrier that opens the cell's level), also the values that are already
// final: the input's Elmore delay, and its driver's arrival and chain length
// unless the driver is on the level just below (still being computed).
template <typename R, int G>
__device__ __forceinline__ void lane_topo(const Topo &t, const State<R> &s, int k, int gl,
                                          LaneTopo<R> &c, bool old_vals) {
    c.k = k;
    c.a = c.b = 0;
    c.has_tv = c.has_old = false;
    if (k < 0) return;
    c.a = ldg(&t.lv_in_ptr[k]);
    c.b = ldg(&t.lv_in_ptr[k + 1]);
    c.e = ldg(&t.lv_onet[k]);
    c.o = ldg(&t.lv_out[k]);
    if (c.b - c.a <= G && gl < c.b - c.a) {
        c.ip = ldg(&t.lv_in_pin[c.a + gl]);
        c.in = ldg(&t.lv_in_net[c.a + gl]);
        c.dv = ldg(&t.lv_in_drv[c.a + gl]);
        c.fl = ldg(&t.lv_in_flags[c.a + gl]);
        if (old_vals) {
            c.tv = ldg(&s.tnet[c.ip]);
            c.has_tv = true;
            if (!(c.fl & kInPrev)) {
                c.ad = ldcg(&s.arr[c.dv]);
                c.pl = ldcg(&s.plen[c.in]);
                c.has_old = true;
            }
        }
    }
}

// Arrival of the group's cell (Section II-B: max over its inputs of the
// driver's arrival plus the Elmore delay, plus the cell delay) and, when
// L > 0, its sidetrack list: lane j holds input j and entry j of the
// inherited list; the own deviations are merged in by rank (an entry's rank
// is the number of entries of both lists before it), and the first L of the
// merged list are written, one aligned block per list.  Every lane of the
// warp calls this (shuffles and ballots span the warp); COH: the drivers'
// values were written by other blocks of the same launch.  Warps whose cells
// all have at most kPre inputs take an unrolled path.
template <typename R, int L, bool COH>
__device__ __forceinline__ void fwd_group(const Topo &t, State<R> &s, const LaneTopo<R> &c, int lane) {
    constexpr int G = list_group(L);
    constexpr unsigned gmask = G == 32 ? 0xffffffffu : ((1u << G) - 1u);
    using AC = Acc<R>;
    using A = typename AC::T;
    const unsigned FULL = 0xffffffffu;
    const int gl = lane & (G - 1), gbase = lane & ~(G - 1);
    const int nin = c.k >= 0 ? c.b - c.a : 0;
    const bool wide = nin > G;
    const bool act = c.k >= 0 && !wide;
    const bool mine = act && gl < nin;
    const bool narrow = __all_sync(FULL, nin <= kPre);
    A av = AC::ninf();
    int pl = 0;
    R dcell = R(0);
    if (mine) {
        const R tv = c.has_tv ? c.tv : ldg(&s.tnet[c.ip]);
        A ad;
        if (c.has_old) {
            ad = c.ad;
            pl = c.pl;
        } else {
            ad = ldd<COH>(&s.arr[c.dv]);
            pl = ldd<COH>(&s.plen[c.in]);
        }
        av = AC::add(ad, tv);
    }
    if (act && gl == 0) dcell = ldg(&s.dnet[c.e]);
    // worst input: largest arrival, lowest pin on ties
    A best = av;
    int bi = mine ? c.ip : -1;
    bool bv = mine;
    int wl = 0;  // lane (in the group) of the worst input
    int bn = -1, bl = 0, bc = 0;
    if (narrow) {
#pragma unroll
        for (int o = 1; o < kPre; o <<= 1) {
            const A oa = shfl_x(best, o);
            const int oi = shfl_x(bi, o);
            const bool ov = shfl_x((int)bv, o) != 0;
            if (ov && (!bv || AC::gt(oa, best) || (!AC::gt(best, oa) && oi < bi))) {
                best = oa;
                bi = oi;
                bv = true;
            }
        }
        best = shfl_idx(best, gbase);
        bi = shfl_idx(bi, gbase);
        bv = shfl_idx((int)bv, gbase) != 0;
        const unsigned wm = (__ballot_sync(FULL, mine && c.ip == bi) >> gbase) & gmask;
        wl = wm ? __ffs(wm) - 1 : 0;
        bn = shfl_idx(c.in, gbase + wl);
        bl = shfl_idx(pl, gbase + wl);
        bc = shfl_idx(c.fl, gbase + wl) & kInComb;
    } else {
        bn = mine ? c.in : -1;
        bl = pl;
        bc = mine ? (c.fl & kInComb) : 0;
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            const A oa = shfl_x(best, o);
            const int oi = shfl_x(bi, o), on = shfl_x(bn, o), ol = shfl_x(bl, o), oc = shfl_x(bc, o);
            const bool ov = shfl_x((int)bv, o) != 0;
            if (ov && (!bv || AC::gt(oa, best) || (!AC::gt(best, oa) && oi < bi))) {
                best = oa;
                bi = oi;
                bn = on;
                bl = ol;
                bc = oc;
                bv = true;
            }
        }
    }
    if (!bv) {
        bi = bn = -1;
        bl = bc = 0;
    }
    if (mine) s.arr[c.ip] = av;
    if (act && gl == 0) {
        s.arr[c.o] = AC::add(best, dcell);
        s.pred_in[c.e] = bi;
        s.pred_net[c.e] = bn;
        s.plen[c.e] = bl + 2;
    }
    if constexpr (L > 0) {
        LEnt<R> inh{r_inf<R>(), kNoneKey};
        if (act && gl < L && bc) inh = lent_of(ldd<COH>(&s.blist[(size_t)bn * G + gl]));
        const bool has_own = mine && c.ip != bi;
        const LEnt<R> own{AC::diff(best, av), ((c.ip < bi ? 0u : 2u) << 29) | (uint32_t)c.ip};
        int inh_rank = gl, own_rank = 0;
        if (narrow) {  // the group's inputs are its lanes 0..nin-1
            unsigned mb = 0u;
#pragma unroll
            for (int u = 0; u < kPre; ++u) {
                const LEnt<R> x{shfl_idx(own.d, gbase + u), shfl_idx(own.key, gbase + u)};
                const bool xv = bv && u < nin && u != wl;
                if (xv && gl < L && lent_before(x, inh)) ++inh_rank;
                if (xv && has_own && u != gl && lent_before(x, own)) ++own_rank;
                const unsigned bb = __ballot_sync(FULL, xv && gl < L && lent_before(inh, x));
                if (gl == u) mb = bb;
            }
            own_rank += __popc((mb >> gbase) & gmask);
        } else {
            bool done = !has_own;
            for (;;) {  // broadcast the group's own deviations one at a time
                const unsigned rem = __ballot_sync(FULL, !done);
                if (rem == 0u) break;
                const unsigned gm = (rem >> gbase) & gmask;
                const bool live = gm != 0u;
                const int src = live ? __ffs(gm) - 1 : 0;
                const LEnt<R> x{shfl_idx(own.d, gbase + src), shfl_idx(own.key, gbase + src)};
                if (live && gl < L && lent_before(x, inh)) ++inh_rank;
                if (live && has_own && gl != src && lent_before(x, own)) ++own_rank;
                const unsigned bb = __ballot_sync(FULL, live && gl < L && lent_before(inh, x));
                if (live && gl == src) {
                    own_rank += __popc((bb >> gbase) & gmask);
                    done = true;
                }
            }
        }
        BEnt<R> *out = s.blist + (size_t)(act ? c.e : 0) * G;
        if (act && gl < L && inh_rank < L) out[inh_rank] = bent_of(inh);
        if (has_own && own_rank < L) out[own_rank] = BEnt<R>{own.d, c.ip};
        const unsigned vi = __ballot_sync(FULL, act && gl < L && inh.key != kNoneKey);
        const unsigned vo = __ballot_sync(FULL, has_own);
        if (act && gl == 0)
            s.bcnt[c.e] = min(L, __popc((vi >> gbase) & gmask) + __popc((vo >> gbase) & gmask));
    }
    if (wide && gl == 0) fwd_cell_wide<R, L, COH>(t, s, c.k, c.a, c.b);
}

// One launch per level (captured in a CUDA graph): a group of lanes per cell.
template <typename R, int L>
__global__ void __launch_bounds__(kLvThreads) k_fwd_level(Topo t, State<R> s, int lo, int hi) {
    constexpr int G = list_group(L), CPW = 32 / G;
    pdl_trigger();
    const int lane = threadIdx.x & 31;
    const int chunk = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (lo + chunk * CPW >= hi) return;  // whole warps only
    const int k = lo + chunk * CPW + lane / G;
    LaneTopo<R> c;
    lane_topo<R, G>(t, s, k < hi ? k : -1, lane & (G - 1), c, false);
    pdl_wait();  // the timing loads read what earlier launches wrote
    fwd_group<R, L, false>(t, s, c, lane);
}

template <typename R>
static void launch_fwd(const Topo &t, const State<R> &s, int lo, int hi, int L, cudaStream_t cs) {
    const int CPW = 32 / list_group(L);
    const int grid = div_up((int64_t)div_up(hi - lo, CPW) * 32, kLvThreads);
    switch (L) {
        case 0: launch_pdl(k_fwd_level<R, 0>, grid, kLvThreads, cs, t, s, lo, hi); break;
        case 3: launch_pdl(k_fwd_level<R, 3>, grid, kLvThreads, cs, t, s, lo, hi); break;
        case 7: launch_pdl(k_fwd_level<R, 7>, grid, kLvThreads, cs, t, s, lo, hi); break;
        case 15: launch_pdl(k_fwd_level<R, 15>, grid, kLvThreads, cs, t, s, lo, hi); break;
        default: launch_pdl(k_fwd_level<R, 31>, grid, kLvThreads, cs, t, s, lo, hi); break;
    }
}

// Single-launch sweeps: one block of kPsThreads per SM (64 registers a
// thread), as many warps in flight as registers allow, since a level is a few
// latency-bound steps per warp; one block per SM keeps the barrier short.
constexpr int kPsThreads = 1024;
constexpr int kFwdBlocksPerSM = 1;
constexpr int kBwdBlocksPerSM = 1;

// The whole forward sweep in one cooperative launch: levels in order, a
// level's cells in chunks of 32 / G (one per warp), chunk j on block
// j mod gridDim (spreading a level over every SM), a grid-wide barrier
// between levels.  Before each barrier a warp loads its first chunk of the
// next level: topology, Elmore delays and the values of drivers two or more
// levels down, so only the values the level below wrote are left after it.
template <typename R, int L>
__global__ void __launch_bounds__(kPsThreads, kFwdBlocksPerSM) k_fwd_sweep(Topo t, State<R> s, GridSync gs) {
    constexpr int G = list_group(L), CPW = 32 / G;
    const int lane = threadIdx.x & 31, grp = lane / G, gl = lane & (G - 1);
    const int w0 = blockIdx.x + (threadIdx.x >> 5) * gridDim.x;  // first chunk of this warp
    const int wstride = (blockDim.x >> 5) * gridDim.x;
    auto topo_of = [&](int l, int chunk, LaneTopo<R> &c, bool old_vals) {
        const int k = ldg(&t.lvl_ptr[l - 1]) + chunk * CPW + grp;
        lane_topo<R, G>(t, s, k < ldg(&t.lvl_ptr[l]) ? k : -1, gl, c, old_vals);
    };
    LaneTopo<R> pre;
    if (t.depth > 0) topo_of(1, w0, pre, false);
    for (int l = 1; l <= t.depth; ++l) {
        const int nch = div_up_dev(ldg(&t.lvl_ptr[l]) - ldg(&t.lvl_ptr[l - 1]), CPW);
        if (w0 < nch) {
            fwd_group<R, L, true>(t, s, pre, lane);
            for (int ch = w0 + wstride; ch < nch; ch += wstride) {
                LaneTopo<R> c;
                topo_of(l, ch, c, false);
                fwd_group<R, L, true>(t, s, c, lane);
            }
        }
        if (l == t.depth) break;
        topo_of(l + 1, w0, pre, true);
        if (!grid_sync(gs, (unsigned)l * gridDim.x)) return;
    }
}

// ----------------------------------------------------------- backward ---

// req / slack of the sinks first, first+step, ... < b of the net driven by
// pin a, NP sinks per round of loads; returns min over them of req(s) - t(s)
// and the driver's arrival in ad.  The first round's topology loads are
// issued before pdl_wait() (level launches); COH: required times of sink
// cells were written by other blocks of the same launch.
template <typename R, int NP, bool COH>
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
    if constexpr (!COH) pdl_wait();  // everything below reads values earlier kernels wrote
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
                    rq[u] = AC::add(ldd<COH>(&s.req[so[u]]), -ldg(&s.dnet[sn[u]]));
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

// A net of at most kBwSmallFanout sinks in slot i of the small-net table,
// on a group of kBwSmallFanout lanes (a sink per lane; slots of -1 pad a
// level's table).  Every lane of the warp calls this.
template <typename R, bool COH>
__device__ __forceinline__ void bwd_small(const Topo &t, State<R> &s, int i, int lane) {
    using AC = Acc<R>;
    using A = typename AC::T;
    const int gl = lane & (kBwSmallFanout - 1);
    const int a = ldg(&t.bw_sa[i]), b = ldg(&t.bw_sb[i]);
    const int p = a + 1 + gl;
    const bool mine = a >= 0 && p < b;
    int kd = 0, so = 0, sn = 0;
    if (mine) {
        kd = ldg(&t.pin_kind[p]);
        so = ldg(&t.sink_out[p]);
        sn = ldg(&t.sink_onet[p]);
    }
    if constexpr (!COH) pdl_wait();  // everything below reads values earlier kernels wrote
    A m = AC::pinf(), ad = AC::pinf();
    if (a >= 0) ad = ldg(&s.arr[a]);
    if (mine) {
        const R tp = ldg(&s.tnet[p]);
        A rq, ap;
        if (kd == PK_ENDPOINT) {
            ap = AC::add(ad, tp);
            rq = acc_from_double<R>(*s.T);
            s.arr[p] = ap;
        } else {
            rq = AC::add(ldd<COH>(&s.req[so]), -ldg(&s.dnet[sn]));
            ap = ldg(&s.arr[p]);
        }
        s.req[p] = rq;
        s.slack[p] = AC::diff(rq, ap);
        m = AC::add(rq, -tp);
    }
#pragma unroll
    for (int o = kBwSmallFanout / 2; o > 0; o >>= 1) {  // min is exact: any order gives the same value
        const A other = shfl_x(m, o);
        if (AC::lt(other, m)) m = other;
    }
    if (a >= 0 && gl == 0) {
        s.req[a] = m;
        s.slack[a] = AC::diff(m, ad);
    }
}

constexpr int kBwNetsPerWarp = 32 / kBwSmallFanout;

// One warp-wide task w of a backward level: w < 8 ns is a chunk of
// kBwNetsPerWarp small nets of the level's ns groups of 32 (from group s_lo);
// after that, piece b_lo + (w - 8 ns) of a larger net (lanes stride its sinks).
template <typename R, bool COH>
__device__ __forceinline__ void bwd_task(const Topo &t, State<R> &s, int w, int s_lo, int ns, int b_lo,
                                         int lane) {
    using AC = Acc<R>;
    using A = typename AC::T;
    const int n_small = ns * (32 / kBwNetsPerWarp);
    if (w < n_small) {
        bwd_small<R, COH>(t, s, s_lo * 32 + w * kBwNetsPerWarp + lane / kBwSmallFanout, lane);
        return;
    }
    const BwTask task = t.bw_task[b_lo + (w - n_small)];
    const int a = task.drv;
    A ad;
    A m = net_sinks_req<R, kPre, COH>(t, s, task.p0 + lane, task.p1, 32, a, ad);
    for (int o = 16; o > 0; o >>= 1) {
        const A other = shfl_x(m, o);
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
        m = ldcg(&s.bw_part[base]);
        for (int j = 1; j < task.nparts; ++j) {
            const A v = ldcg(&s.bw_part[base + j]);
            if (AC::lt(v, m)) m = v;
        }
    }
    s.req[a] = m;
    s.slack[a] = AC::diff(m, ad);
}

// warp tasks of a backward level
__host__ __device__ __forceinline__ int bwd_tasks(int ns, int nb) {
    return ns * (32 / kBwNetsPerWarp) + nb;
}

// One launch per level (captured in a CUDA graph): a warp per task.
template <typename R>
__global__ void __launch_bounds__(kLvThreads) k_bwd_level(Topo t, State<R> s, int s_lo, int ns,
                                                          int b_lo, int nb) {
    pdl_trigger();
    const int w = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (w >= bwd_tasks(ns, nb)) return;
    bwd_task<R, false>(t, s, w, s_lo, ns, b_lo, threadIdx.x & 31);
}

// ---------------------------------------------------------- WNS / TNS ---

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 148;
constexpr int kCoopMaxBlocks = 1024;  // cap on the grid of a cooperative launch

// WNS = min over endpoints with negative slack, TNS = their sum (FP64;
// Eqs. (3)-(4)).  The endpoints are cut into chunks of kRedChunk, a warp
// reduces one chunk in a fixed order, and the last block to finish adds the
// chunk partials in chunk order: the result does not depend on the grid, the
// block size or scheduling.
template <typename R, bool COH>
__device__ __forceinline__ void wns_tns_blocks(const Topo &t, State<R> &s) {
    __shared__ bool last;
    const int lane = threadIdx.x & 31;
    const int n_chunks = div_up_dev(t.n_ep, kRedChunk);
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int ch = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); ch < n_chunks; ch += nw) {
        double mn = 0.0, sm = 0.0;
        const int end = min((ch + 1) * kRedChunk, t.n_ep);
        for (int i = ch * kRedChunk + lane; i < end; i += 32) {
            const double v = (double)ldd<COH>(&s.slack[ldg(&t.ep[i])]);
            if (v < 0.0) {
                mn = fmin(mn, v);
                sm += v;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
            sm += __shfl_xor_sync(0xffffffffu, sm, o);
        }
        if (lane == 0) {
            s.red_part[2 * ch] = mn;
            s.red_part[2 * ch + 1] = sm;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(s.red_count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double bm = 0.0, bs = 0.0;
        for (int k = 0; k < n_chunks; ++k) {
            bm = fmin(bm, ldcg(&s.red_part[2 * k]));
            bs += ldcg(&s.red_part[2 * k + 1]);
        }
        s.wns_tns[0] = bm;
        s.wns_tns[1] = bs;
        *s.red_count = 0u;
    }
}

template <typename R>
__global__ void __launch_bounds__(kRedThreads) k_wns_tns(Topo t, State<R> s) {
    pdl_wait();
    wns_tns_blocks<R, false>(t, s);
}

// The whole backward sweep and WNS / TNS in one cooperative launch: levels
// from the deepest down to the startpoints' nets, tasks of a level spread
// over all warps, a grid-wide barrier after each level.
template <typename R>
__global__ void __launch_bounds__(kPsThreads, kBwdBlocksPerSM) k_bwd_sweep(Topo t, State<R> s, GridSync gs) {
    const int lane = threadIdx.x & 31;
    const int w0 = blockIdx.x + (threadIdx.x >> 5) * gridDim.x;  // task j on block j mod gridDim
    const int wstride = (blockDim.x >> 5) * gridDim.x;
    unsigned n = 0;
    for (int l = t.depth; l >= 0; --l) {
        const int4 q = ldg(&t.bw_lv[l]);  // small groups (first, count), pieces (first, count)
        const int nt = bwd_tasks(q.y, q.w);
        for (int w = w0; w < nt; w += wstride) bwd_task<R, true>(t, s, w, q.x, q.y, q.z, lane);
        if (!grid_sync(gs, (++n) * gridDim.x)) return;
    }
    wns_tns_blocks<R, true>(t, s);
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
            launch_pdl(k_bwd_level<R>, div_up((int64_t)bwd_tasks(ns, nb) * 32, kLvThreads), kLvThreads, cs, t, s,
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

// Blocks of a cooperative launch of `kernel` that are resident at once (at
// most kCoopMaxBlocks), cached per kernel; 0 if none.
template <typename K>
static int coop_grid(tdp_graph *g, K kernel) {
    const void *key = reinterpret_cast<const void *>(kernel);
    for (auto &pr : g->coop_grid)
        if (pr.first == key) return pr.second;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, kPsThreads, 0) != cudaSuccess) {
        cudaGetLastError();
        nb = 0;
    }
    const int grid = std::min(nb * g->n_sm, kCoopMaxBlocks);
    g->coop_grid.emplace_back(key, grid);
    return grid;
}

template <typename R>
static tdp_status launch_sweep(tdp_graph *g, void (*kernel)(Topo, State<R>, GridSync), int grid,
                               KernelId id) {
    State<R> &s = state<R>(g);
    GridSync gs;
    gs.count = s.gsync;
    gs.status = s.gsync + 1;
    gs.timeout_ns = kSyncTimeoutNs;
    LaunchScope ls(g, id);
    TDP_CUDA(cudaMemsetAsync(s.gsync, 0, sizeof(unsigned), g->stream));
    TDP_CUDA(launch_coop(kernel, grid, kPsThreads, g->stream, g->topo, s, gs));
    return TDP_OK;
}

// Forward sweep, building sidetrack lists of length g->list_L (0: none): one
// cooperative launch, or one graph replay of the level launches.  Run again,
// it writes the same arrival times.
template <typename R>
tdp_status forward_lists(tdp_graph *g) {
    State<R> &s = state<R>(g);
    if (g->list_L > 0 && !s.blist) TDP_TRY(dalloc(g, &s.blist, (size_t)g->topo.n_nets * kMaxK));
    if (g->single_launch) {
        if (g->topo.depth == 0) return TDP_OK;
        void (*kernel)(Topo, State<R>, GridSync);
        switch (g->list_L) {
            case 0: kernel = k_fwd_sweep<R, 0>; break;
            case 3: kernel = k_fwd_sweep<R, 3>; break;
            case 7: kernel = k_fwd_sweep<R, 7>; break;
            case 15: kernel = k_fwd_sweep<R, 15>; break;
            default: kernel = k_fwd_sweep<R, 31>; break;
        }
        const int grid = coop_grid(g, kernel);
        if (grid > 0) return launch_sweep<R>(g, kernel, grid, KID_FWD_SWEEP);
        g->single_launch = false;  // no resident grid: per-level launches from now on
    }
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

// Backward sweep and WNS / TNS: one cooperative launch, or one graph replay.
template <typename R>
static tdp_status backward(tdp_graph *g) {
    if (g->single_launch) {
        const int grid = coop_grid(g, k_bwd_sweep<R>);
        if (grid > 0) return launch_sweep<R>(g, k_bwd_sweep<R>, grid, KID_BWD_SWEEP);
        g->single_launch = false;
    }
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
    if (g->list_L > 0 && !s.blist) TDP_TRY(dalloc(g, &s.blist, (size_t)t.n_nets * kMaxK));
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
        TDP_TRY(check_sync_status(g));  // synchronises the stream
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
