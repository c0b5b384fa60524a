// Pin-pair set P and weights, Eq. (w_ij) (Section III-D).
//
// k_pair_walk walks every extracted path (thread per path) and, for every
// net arc (driver -> sink s) on it, adds q = slack / WNS of the path to the
// accumulators of s and raises the running maximum of q at s.  Both are kept
// as 64-bit fixed point (2^-24), so the integer atomics are exact and the
// result does not depend on the order of the paths.
//
// k_pair_finish applies the rule to every touched sink (one whose maximum a
// walk raised above its initial LLONG_MIN).  Traversing the paths
// worst first, the first path through a new pair sets w0 and every later one
// adds w1 * q; the first one is the path with the largest q (most negative
// slack), so
//     new pair:      w = w0 + w1 * (sum q - max q)
//     pair in P:     w = w  + w1 * sum q.
#include <algorithm>
#include <climits>

#include "tdp_internal.cuh"

namespace tdp {

constexpr int kWalkWarps = 4;

// A warp takes 32 / KP failing endpoints (KP: K rounded up to a power of
// two); lane g * KP + r walks the path of rank r of the warp's endpoint g
// from the endpoint back to its startpoint, one net arc per step.  Paths of
// one endpoint share their first arcs, and lanes standing on the same sink
// in the same step are merged (__match_any_sync): the lowest such lane adds
// the group's summed q and raises the maximum once for all of them (sums and
// maxima do not depend on how the lanes are grouped).
// (at most 32 registers a thread: beside a block of the backward sweep an SM
// then holds four blocks of this kernel instead of three)
template <typename R>
__global__ void __launch_bounds__(kWalkWarps * 32, 16) k_pair_walk(Topo t, State<R> s, int K, int KP, int n_cap) {
    __shared__ long long shQ[kWalkWarps][32];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int per = 32 / KP, g = lane / KP, r = lane % KP;
    chain_enter();
    const int nv = min(*s.nviol, n_cap);
    const double wns = s.wns_tns[0];
    if (!(wns < 0.0)) return;
    const int n_tasks = (nv + per - 1) / per;
    for (int task = blockIdx.x * kWalkWarps + w; task < n_tasks; task += gridDim.x * kWalkWarps) {
        const int i = task * per + g;
        const bool have = i < nv;
        const int ep = have ? s.viol[i] : -1;
        const int cnt = have ? s.p_count[i] : 0;
        const bool on = r < cnt;
        const size_t base = (size_t)(have ? i : 0) * K;
        long long Q = 0;
        int sides[kMaxK];
        int ns = 0;
        if (on) {
            const R sigma = s.slack[ep] + s.p_cost[base + r];
            double q = (double)sigma / wns;
            q = fmin(fmax(q, -kQClamp), kQClamp);
            Q = __double2ll_rn(q * kQScale);
            for (int x = r; x > 0; x = s.p_parent[base + x]) sides[ns++] = s.p_side[base + x];
        }
        shQ[w][lane] = Q;
        __syncwarp();
        // the endpoint's own net arc is on every path of the endpoint
        if (r == 0 && have) {
            long long sum = 0, mx = LLONG_MIN;
            for (int l = 0; l < cnt; ++l) {
                sum += shQ[w][g * KP + l];
                mx = max(mx, shQ[w][g * KP + l]);
            }
            atomicAdd((unsigned long long *)&s.sumq[ep], (unsigned long long)sum);
            atomicMax(&s.maxq[ep], mx);
        }
        int e = on ? t.pin_net[ep] : 0;
        int j = ns - 1;  // sides[] holds the deepest sidetrack first
        // the next sidetrack to take, in registers: its pin, the net where
        // it is taken (-2: none) and the net it leads to; refreshed only
        // when it is taken, so that a step's only dependent load is pred
        int nside = -1, nat = -2, nto = -1;
        auto next_side = [&]() {
            if (j >= 0) {
                nside = sides[j];
                nat = t.sink_onet[nside];
                nto = t.pin_net[nside];
            } else {
                nat = -2;
            }
        };
        next_side();
        bool walking = on;
        unsigned last_mask = 0;
        long long last_sum = 0, last_max = 0;
        for (;;) {
            int pin = -1 - lane;  // distinct per lane when not on a sink
            if (walking) {
                const int2 pr = s.pred[e];
                int pi = pr.x;
                if (pi < 0) {
                    walking = false;
                } else {
                    int nx;
                    if (nat == e) {
                        pi = nside;
                        nx = nto;
                        --j;
                        next_side();
                    } else {
                        nx = pr.y;
                    }
                    pin = pi;
                    e = nx;
                }
            }
            if (!__any_sync(FULL, walking)) break;
            const unsigned grp = __match_any_sync(FULL, pin);
            if (walking && lane == __ffs(grp) - 1) {
                if (grp != last_mask) {
                    last_sum = 0;
                    last_max = LLONG_MIN;
                    for (unsigned m = grp; m; m &= m - 1) {
                        const long long v = shQ[w][__ffs(m) - 1];
                        last_sum += v;
                        last_max = max(last_max, v);
                    }
                    last_mask = grp;
                }
                atomicAdd((unsigned long long *)&s.sumq[pin], (unsigned long long)last_sum);
                atomicMax(&s.maxq[pin], last_max);
            }
        }
        __syncwarp();
    }
}

// The update of one touched sink p not yet in P (the rule above): it joins
// P with w = w0 + w1 * (sum q - max q), and its net and cells get the loss's
// flags.
template <typename R>
__device__ __forceinline__ void pair_new(const Topo &t, State<R> &s, int p, long long mx, double w0, double w1) {
    const double sq = (double)s.sumq[p] / kQScale;
    const double mq = (double)mx / kQScale;
    s.w[p] = (R)(w0 + w1 * (sq - mq));
    s.in_p[p] = 1;
    atomicAdd((unsigned long long *)s.n_pairs, 1ull);
    // flags for the loss lists (set only; threads of one net write the same value)
    const int e = t.pin_net[p];
    const int a = t.net_ptr[e];
    s.net_pf[e] = t.net_ptr[e + 1] - a - 1 <= kBigFanout ? kPfSmall : kPfLarge;
    s.cell_pf[t.pin_cell[p]] = 1;
    s.cell_pf[t.pin_cell[a]] = 1;
    s.sumq[p] = 0;
    s.maxq[p] = LLONG_MIN;
}

// The rule on every touched sink, in one launch with two roles on disjoint
// sinks.  Blocks [0, p_blocks) take the sinks already in P from the list of
// the last compaction (a thread a listed sink, so that the FP64 arithmetic
// runs on dense warps): w += w1 * sum q.  The other blocks scan every pin's
// maximum, two a 16-byte load, kFinishLoads loads issued before a thread
// looks at any: a sink is touched when a walk raised its maximum (every q is
// finite), and a touched sink not in P is new.  A sink in P is left to the
// first role whichever of its maxima the scan reads (in_p does not change
// for it here), so no sink is updated twice.
constexpr int kFinishLoads = 4;
template <typename R>
__global__ void k_pair_finish(Topo t, State<R> s, int n_pins, double w0, double w1, int p_blocks) {
    chain_enter();
    if ((int)blockIdx.x < p_blocks) {
        const int np = s.pcnt[0];
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += p_blocks * blockDim.x) {
            const int p = s.ppins[i];
            if (s.maxq[p] == LLONG_MIN) continue;
            const double sq = (double)s.sumq[p] / kQScale;
            s.w[p] = (R)((double)s.w[p] + w1 * sq);
            s.sumq[p] = 0;
            s.maxq[p] = LLONG_MIN;
        }
        return;
    }
    const int bid = (int)blockIdx.x - p_blocks;
    const longlong2 *m2 = reinterpret_cast<const longlong2 *>(s.maxq);
    const int half = n_pins / 2;
    const int stride = ((int)gridDim.x - p_blocks) * blockDim.x;
    for (int i0 = bid * blockDim.x + threadIdx.x; i0 < half; i0 += kFinishLoads * stride) {
        longlong2 m[kFinishLoads];
#pragma unroll
        for (int u = 0; u < kFinishLoads; ++u) {
            const int i = i0 + u * stride;
            m[u] = i < half ? __ldcg(m2 + i) : make_longlong2(LLONG_MIN, LLONG_MIN);
        }
#pragma unroll
        for (int u = 0; u < kFinishLoads; ++u) {
            const int i = i0 + u * stride;
            if (m[u].x != LLONG_MIN && !s.in_p[2 * i]) pair_new(t, s, 2 * i, m[u].x, w0, w1);
            if (m[u].y != LLONG_MIN && !s.in_p[2 * i + 1]) pair_new(t, s, 2 * i + 1, m[u].y, w0, w1);
        }
    }
    if ((n_pins & 1) && bid == 0 && threadIdx.x == 0) {
        const long long m = __ldcg(&s.maxq[n_pins - 1]);
        if (m != LLONG_MIN && !s.in_p[n_pins - 1]) pair_new(t, s, n_pins - 1, m, w0, w1);
    }
}

// ------------------------------------------------------- compaction ---
// Indices i < n with flag[i] == val, ascending (k_compact, below).  A
// thread takes 32 consecutive flags (two 16-byte loads), a block a tile of
// kCompactItems.

constexpr int kCmpThreads = kCompactItems / 32;

__device__ __forceinline__ unsigned match_bits(const uint8_t *f, int base, int n, uint8_t val) {
    unsigned bits = 0u;
    if (base + 32 <= n) {
        const uint4 *v = reinterpret_cast<const uint4 *>(f + base);
        const uint4 q0 = __ldg(v), q1 = __ldg(v + 1);
        const unsigned w[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
#pragma unroll
        for (int k = 0; k < 32; ++k)
            if (((w[k >> 2] >> (8 * (k & 3))) & 0xffu) == val) bits |= 1u << k;
    } else {
        for (int k = 0; k < 32 && base + k < n; ++k)
            if (f[base + k] == val) bits |= 1u << k;
    }
    return bits;
}

__device__ __forceinline__ int block_excl_sum(int v, int *sh, int &total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        int t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        sh[lane] = t;
    }
    __syncthreads();
    total = sh[(blockDim.x >> 5) - 1];
    const int before = (w > 0 ? sh[w - 1] : 0) + x - v;
    __syncthreads();
    return before;
}

// One pass (decoupled look-back): a block takes the next tile of
// kCompactItems flags from a counter, so every earlier tile belongs to a
// block that is running or done; it counts its matches, publishes the
// count, adds the counts of the tiles before it back to the first that has
// published its inclusive prefix, publishes its own inclusive prefix and
// writes its indices.  Two flag arrays share a launch as two runs of tiles;
// a look-back ends at the first tile of its own run.  A tile's state is one
// 64-bit word: the call's epoch (30 bits, so that nothing is cleared between
// calls), a flag (count / inclusive prefix) and the value.  The last block
// to finish resets the counters for the next call.  A look-back that polls
// too long (2^22 polls) sets the graph's sticky status (reported as
// TDP_ERR_TIMEOUT) and stops.
constexpr unsigned kCmpAgg = 1u, kCmpIncl = 2u;
__device__ __forceinline__ unsigned long long cmp_word(unsigned epoch, unsigned flag, unsigned v) {
    return ((unsigned long long)(epoch & 0x3fffffffu) << 34) | ((unsigned long long)flag << 32) | v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// The sum of the counts of tiles first .. tile - 1, by one warp: it reads the
// states of the 32 tiles below j at once (lane l reads tile j - l) and, once
// every tile down to the nearest inclusive prefix has published, adds their
// values; without an inclusive prefix in the window it moves down 32 tiles.
// A tile below first reads as an inclusive prefix of 0.
__device__ __forceinline__ int cmp_look_back(unsigned long long *tiles, int tile, int first, unsigned epoch,
                                             unsigned *status) {
    const int lane = threadIdx.x & 31;
    const unsigned ep = epoch & 0x3fffffffu;
    int prefix = 0;
    unsigned polls = 0;
    for (int j = tile - 1;;) {
        const int jj = j - lane;
        unsigned flag = kCmpIncl, v = 0u;
        if (jj >= first) {
            const unsigned long long w = ld_relaxed_u64(&tiles[jj]);
            flag = (unsigned)(w >> 34) == ep ? (unsigned)(w >> 32) & 3u : 0u;
            v = (unsigned)w;
        }
        const unsigned incl = __ballot_sync(0xffffffffu, flag == kCmpIncl);
        const unsigned wait = __ballot_sync(0xffffffffu, flag == 0u);
        const int stop = incl ? __ffs(incl) - 1 : 31;  // the last lane the sum takes
        const unsigned need = stop == 31 ? 0xffffffffu : (2u << stop) - 1u;
        if (wait & need) {
            if (++polls > (1u << 22)) {
                if (lane == 0) atomicExch(status, 1u);
                break;
            }
            continue;
        }
        int x = lane <= stop ? (int)v : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        prefix += x;
        if (incl) break;
        j -= 32;
    }
    return prefix;
}

__global__ void __launch_bounds__(kCmpThreads) k_compact(CmpPart p0, CmpPart p1, int nb0, int nb,
                                                        unsigned long long *tiles, unsigned *ctr, unsigned epoch,
                                                        unsigned *status, int32_t *clear32, long long *clear64) {
    __shared__ int sh[32];
    __shared__ int s_tile, s_prefix;
    chain_enter();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (clear32) *clear32 = 0;
        if (clear64) *clear64 = 0;
    }
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(&ctr[0], 1u);
    __syncthreads();
    const int tile = s_tile;
    if (tile >= nb) {  // the counters were not reset: no tile state to touch
        if (threadIdx.x == 0) {
            atomicExch(status, 1u);
            if (atomicAdd(&ctr[1], 1u) == (unsigned)nb - 1u) {
                ctr[0] = 0u;
                ctr[1] = 0u;
            }
        }
        return;
    }
    const bool second = tile >= nb0;
    const CmpPart p = second ? p1 : p0;
    const int first = second ? nb0 : 0, last = second ? nb - 1 : nb0 - 1;
    const int base = (tile - first) * kCompactItems + threadIdx.x * 32;
    unsigned bits = match_bits(p.f, base, p.n, p.val);
    int total;
    const int before = block_excl_sum(__popc(bits), sh, total);
    if (threadIdx.x < 32) {
        if (tile > first && threadIdx.x == 0) st_relaxed_u64(&tiles[tile], cmp_word(epoch, kCmpAgg, (unsigned)total));
        const int prefix = tile > first ? cmp_look_back(tiles, tile, first, epoch, status) : 0;
        if (threadIdx.x == 0) {
            st_relaxed_u64(&tiles[tile], cmp_word(epoch, kCmpIncl, (unsigned)(prefix + total)));
            s_prefix = prefix;
            if (tile == last) *p.count = prefix + total;
        }
    }
    __syncthreads();
    int pos = s_prefix + before;
    while (bits) {
        const int k = __ffs(bits) - 1;
        p.out[pos++] = p.map ? p.map[base + k] : base + k;
        bits &= bits - 1u;
    }
    if (threadIdx.x == 0 && atomicAdd(&ctr[1], 1u) == (unsigned)nb - 1u) {
        ctr[0] = 0u;
        ctr[1] = 0u;
    }
}

tdp_status compact_flags(tdp_graph *g, const CmpPart &a, const CmpPart *b, int32_t *clear32, long long *clear64) {
    unsigned long long *tiles = g->prec == TDP_FP32 ? g->s32.cmp_tiles : g->s64.cmp_tiles;
    unsigned *ctr = g->prec == TDP_FP32 ? g->s32.cmp_ctr : g->s64.cmp_ctr;
    unsigned *status = g->prec == TDP_FP32 ? g->s32.gsync + 1 : g->s64.gsync + 1;
    const int nb0 = std::max(div_up(a.n, kCompactItems), 1);
    const int nb = nb0 + (b ? std::max(div_up(b->n, kCompactItems), 1) : 0);
    if ((size_t)nb > compact_tile_cap(g->topo)) {
        set_error("compaction: %d tiles, %zu tile states", nb, compact_tile_cap(g->topo));
        return TDP_ERR_INVALID;
    }
    const unsigned epoch = ++g->cmp_epoch;
    TDP_CUDA(launch_pdl(k_compact, nb, kCmpThreads, g->stream, a, b ? *b : a, nb0, nb, tiles, ctr, epoch, status,
                        clear32, clear64));
    return TDP_OK;
}

// The loss's pair records (State::pr_*), a thread per sink of P: what the
// loss passes read per pair in two rounds of loads (the record, then the two
// cells' positions) instead of walking pin -> net -> driver -> cell.  The
// first pair of a net finds the net's pairs (the records are ascending by
// pin, and the net's pins end at net_ptr[e + 1]) by a binary search over at
// most the net's fanout records.
template <typename R>
__global__ void k_pair_records(Topo t, State<R> s) {
    chain_enter();
    const int np = s.pcnt[0];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
        const int p = s.ppins[i];
        const int e = t.pin_net[p];
        const int a = t.net_ptr[e], b = t.net_ptr[e + 1];
        const bool big = b - a - 1 > kBigFanout;
        int dslot = -1;
        if (i == 0 || t.pin_net[s.ppins[i - 1]] != e) {
            int lo = i + 1, hi = min(np, i + (b - a - 1));
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (s.ppins[mid] < b) lo = mid + 1;
                else hi = mid;
            }
            const int cnt = lo - i;
            s.pr_n[i] = cnt;
            if (big) s.pr_big[atomicAdd(s.pr_nbig, 1)] = make_int4(i, cnt, t.slot_of_pin[a], 0);
            else dslot = t.slot_of_pin[a];
        }
        s.pr_a[i] = make_int4(t.pin_cell[p], t.pin_cell[a], t.slot_of_pin[p], dslot);
        R *o = s.pr_o + 4 * (size_t)i;
        o[0] = s.pin_dx[p];
        o[1] = s.pin_dy[p];
        o[2] = s.pin_dx[a];
        o[3] = s.pin_dy[a];
        s.pr_w[i] = s.w[p];
    }
}

template <typename R>
tdp_status compact_pairs(tdp_graph *g) {
    const Topo &t = g->topo;
    State<R> &s = state<R>(g);
    const CmpPart cells{s.cell_pf, nullptr, s.pcells, s.pcnt + 1, t.n_cells, 1};
    TDP_TRY(compact_flags(g, CmpPart{s.in_p, nullptr, s.ppins, s.pcnt, t.n_pins, 1}, &cells, s.pr_nbig));
    TDP_CUDA(launch_pdl(k_pair_records<R>, 148 * 4, 256, g->stream, t, s));
    g->n_launch += 2;
    return TDP_OK;
}

template tdp_status compact_pairs<float>(tdp_graph *);
template tdp_status compact_pairs<double>(tdp_graph *);

template <typename R>
tdp_status update_pairs_impl(tdp_graph *g, double w0, double w1) {
    Topo &t = g->topo;
    State<R> &s = state<R>(g);
    const int n_cap = g->n_endpoints < 0 ? INT_MAX : g->n_endpoints;
    if (g->rt_mode) {
        rt_pair_walk<R>(g);
    } else if (t.n_ep > 0) {
        LaunchScope ls(g, KID_PAIR_WALK);
        int KP = 1;
        while (KP < g->K) KP *= 2;
        const int blocks = std::min(div_up(div_up(t.n_ep, 32 / KP), kWalkWarps), 148 * 16);
        TDP_CUDA(launch_pdl(k_pair_walk<R>, blocks, kWalkWarps * 32, g->stream, t, s, g->K, KP, n_cap));
    }
    {
        LaunchScope ls(g, KID_PAIR_FINISH);
        constexpr int p_blocks = 148 * 2;
        TDP_CUDA(launch_pdl(k_pair_finish<R>, p_blocks + 148 * 8, 256, g->stream, t, s, t.n_pins, w0, w1, p_blocks));
    }
    return compact_pairs<R>(g);
}

template tdp_status update_pairs_impl<float>(tdp_graph *, double, double);
template tdp_status update_pairs_impl<double>(tdp_graph *, double, double);

// ------------------------------------------------------------ get / set ---

template <typename R>
__global__ void k_flag_in_p(const State<R> s, int n, int32_t *flags) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) flags[p] = s.in_p[p] ? 1 : 0;
}

template <typename R>
__global__ void k_scatter_pairs(const State<R> s, int n, const int64_t *off, int32_t *pins, R *w) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n || !s.in_p[p]) return;
    int64_t k = off[p];
    if (pins) pins[k] = p;
    if (w) w[k] = s.w[p];
}

template <typename R>
static tdp_status get_pairs_impl(tdp_graph *g, int32_t *pins, R *w, int64_t *n_out) {
    State<R> &s = state<R>(g);
    const int n = g->topo.n_pins;
    cudaStream_t st = g->stream;
    int32_t *flags = nullptr;
    int64_t *off = nullptr;
    if (dmalloc_async(&flags, sizeof(int32_t) * n, st) != cudaSuccess ||
        dmalloc_async(&off, sizeof(int64_t) * (n + 1), st) != cudaSuccess) {
        if (flags) cudaFreeAsync(flags, st);
        set_error("attraction_get_pairs: temporary allocation failed");
        return TDP_ERR_OOM;
    }
    g->n_launch += 2;
    k_flag_in_p<R><<<div_up(n, 256), 256, 0, st>>>(s, n, flags);
    tdp_status rc = scan_i32_to_i64(g, flags, off, n, st);
    if (rc == TDP_OK && (pins || w)) k_scatter_pairs<R><<<div_up(n, 256), 256, 0, st>>>(s, n, off, pins, w);
    int64_t total = 0;
    if (rc == TDP_OK) {
        cudaMemcpyAsync(&total, off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) {
            set_error("attraction_get_pairs: %s", cudaGetErrorString(cudaGetLastError()));
            rc = TDP_ERR_CUDA;
        }
    }
    cudaFreeAsync(flags, st);
    cudaFreeAsync(off, st);
    if (n_out) *n_out = total;
    return rc;
}

template <typename R>
static tdp_status set_pairs_impl(tdp_graph *g, int64_t n, const int32_t *pins, const double *w) {
    State<R> &s = state<R>(g);
    const int np = g->topo.n_pins;
    std::vector<uint8_t> in_p(np, 0);
    std::vector<R> wv(np, R(0));
    std::vector<int32_t> pn(np);
    // sinks are all pins that are not the first pin of their net
    std::vector<uint8_t> is_sink(np, 1);
    {
        std::vector<int32_t> ptr(g->topo.n_nets + 1);
        TDP_CUDA(cudaMemcpy(ptr.data(), g->topo.net_ptr, sizeof(int32_t) * ptr.size(), cudaMemcpyDeviceToHost));
        for (int e = 0; e < g->topo.n_nets; ++e) is_sink[ptr[e]] = 0;
    }
    for (int64_t k = 0; k < n; ++k) {
        int p = pins[k];
        if (p < 0 || p >= np || !is_sink[p] || in_p[p] || !std::isfinite(w[k])) {
            set_error("attraction_set_pairs: entry %lld (pin %d) is not a distinct sink pin with a "
                      "finite weight", (long long)k, p);
            return TDP_ERR_INVALID;
        }
        in_p[p] = 1;
        wv[p] = (R)w[k];
    }
    // loss flags: nets holding a pair sink, cells of pair sinks and of their drivers
    const Topo &t = g->topo;
    std::vector<int32_t> ptr(t.n_nets + 1), pcell(np);
    TDP_CUDA(cudaMemcpy(ptr.data(), t.net_ptr, sizeof(int32_t) * ptr.size(), cudaMemcpyDeviceToHost));
    TDP_CUDA(cudaMemcpy(pcell.data(), t.pin_cell, sizeof(int32_t) * np, cudaMemcpyDeviceToHost));
    std::vector<uint8_t> npf(t.n_nets, 0), cpf(t.n_cells, 0);
    for (int e = 0; e < t.n_nets; ++e)
        for (int p = ptr[e] + 1; p < ptr[e + 1]; ++p)
            if (in_p[p]) {
                npf[e] = ptr[e + 1] - ptr[e] - 1 <= kBigFanout ? kPfSmall : kPfLarge;
                cpf[pcell[p]] = 1;
                cpf[pcell[ptr[e]]] = 1;
            }
    long long cnt = n;
    TDP_CUDA(cudaStreamSynchronize(g->stream));
    TDP_CUDA(cudaMemcpy(s.in_p, in_p.data(), np, cudaMemcpyHostToDevice));
    TDP_CUDA(cudaMemcpy(s.w, wv.data(), sizeof(R) * np, cudaMemcpyHostToDevice));
    TDP_CUDA(cudaMemcpy(s.n_pairs, &cnt, sizeof(cnt), cudaMemcpyHostToDevice));
    TDP_CUDA(cudaMemcpy(s.net_pf, npf.data(), t.n_nets, cudaMemcpyHostToDevice));
    TDP_CUDA(cudaMemcpy(s.cell_pf, cpf.data(), t.n_cells, cudaMemcpyHostToDevice));
    TDP_CUDA(cudaMemset(s.gslot, 0, 2 * sizeof(R) * (size_t)np));
    return compact_pairs<R>(g);
}

template <typename R>
static tdp_status reset_pairs_impl(tdp_graph *g) {
    State<R> &s = state<R>(g);
    const int np = g->topo.n_pins;
    TDP_CUDA(cudaMemsetAsync(s.in_p, 0, np, g->stream));
    TDP_CUDA(cudaMemsetAsync(s.w, 0, sizeof(R) * np, g->stream));
    TDP_CUDA(cudaMemsetAsync(s.n_pairs, 0, sizeof(long long), g->stream));
    TDP_CUDA(cudaMemsetAsync(s.net_pf, 0, g->topo.n_nets, g->stream));
    TDP_CUDA(cudaMemsetAsync(s.cell_pf, 0, g->topo.n_cells, g->stream));
    TDP_CUDA(cudaMemsetAsync(s.pcnt, 0, 2 * sizeof(int32_t), g->stream));
    TDP_CUDA(cudaMemsetAsync(s.pr_nbig, 0, sizeof(int32_t), g->stream));
    TDP_CUDA(cudaMemsetAsync(s.gslot, 0, 2 * sizeof(R) * (size_t)np, g->stream));
    return TDP_OK;
}

}  // namespace tdp

using namespace tdp;

extern "C" tdp_status attraction_update_pairs(tdp_graph *g, double w0, double w1,
                                              int64_t *n_pairs_out) {
    if (!g || !std::isfinite(w0) || !std::isfinite(w1)) {
        set_error("attraction_update_pairs: NULL graph or non-finite w0 / w1");
        return TDP_ERR_INVALID;
    }
    if (!g->extracted) {
        set_error("attraction_update_pairs: call extract_critical_paths first");
        return TDP_ERR_STATE;
    }
    tdp_status st = g->prec == TDP_FP32 ? update_pairs_impl<float>(g, w0, w1)
                                        : update_pairs_impl<double>(g, w0, w1);
    if (st != TDP_OK) return st;
    if (n_pairs_out) {
        long long h = 0;
        const long long *src = g->prec == TDP_FP32 ? g->s32.n_pairs : g->s64.n_pairs;
        TDP_CUDA(cudaMemcpyAsync(&h, src, sizeof(h), cudaMemcpyDeviceToHost, g->stream));
        TDP_CUDA(cudaStreamSynchronize(g->stream));
        *n_pairs_out = h;
    }
    return TDP_OK;
}

extern "C" tdp_status attraction_reset_pairs(tdp_graph *g) {
    if (!g) {
        set_error("attraction_reset_pairs: NULL graph");
        return TDP_ERR_INVALID;
    }
    return g->prec == TDP_FP32 ? reset_pairs_impl<float>(g) : reset_pairs_impl<double>(g);
}

extern "C" tdp_status attraction_set_pairs(tdp_graph *g, int64_t n_pairs, const int32_t *pins_host,
                                           const double *w_host) {
    if (!g || n_pairs < 0 || (n_pairs > 0 && (!pins_host || !w_host))) {
        set_error("attraction_set_pairs: NULL graph or arrays, or negative count");
        return TDP_ERR_INVALID;
    }
    return g->prec == TDP_FP32 ? set_pairs_impl<float>(g, n_pairs, pins_host, w_host)
                               : set_pairs_impl<double>(g, n_pairs, pins_host, w_host);
}

extern "C" tdp_status attraction_get_pairs(tdp_graph *g, int32_t *pins_dev, void *w_dev,
                                           int64_t *n_pairs_out) {
    if (!g) {
        set_error("attraction_get_pairs: NULL graph");
        return TDP_ERR_INVALID;
    }
    return g->prec == TDP_FP32 ? get_pairs_impl<float>(g, pins_dev, (float *)w_dev, n_pairs_out)
                               : get_pairs_impl<double>(g, pins_dev, (double *)w_dev, n_pairs_out);
}
