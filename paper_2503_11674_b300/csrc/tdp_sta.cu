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
//   k_ep_wns     endpoints: arrival, required time (T), slack and the
//                failing flag, and WNS / TNS over them (FP64, fixed-order
//                reduction); they need the forward sweep only
//   k_bwd_sweep  the backward sweep in one cooperative launch: required times
//                of the nets driven from each level, deepest first (a net of
//                at most 8 sinks on an aligned group of 1, 2 or 4 lanes, a
//                warp per 64-sink piece of a larger net, the pieces combined
//                by an atomic min on an order-preserving key).  Required
//                times need no arrival, and nothing later in a timing
//                iteration reads them, so it runs on a second stream
//                beside path extraction, the pair update and the loss
//   k_pin_req, k_in_arr, k_pin_slack
//                required time, input-pin arrival and slack of every pin
//                that is not an endpoint, on request (sta_get_timing)
//
// Where a cooperative launch cannot be made resident (or TDP_LEVEL_GRAPHS=1),
// the same per-cell and per-task code runs as one launch per level
// (k_fwd_level, k_bwd_level) captured in CUDA graphs; there every
// array a level reads was written by an earlier launch, so the reads use the
// read-only path.  Inside one cooperative launch, values written before a
// barrier are read from L2.  Either way all loads of a group of inputs /
// sinks are issued before the first store.
#include <algorithm>
#include <climits>
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

__device__ __forceinline__ bool same_bits(float a, float b) { return __float_as_uint(a) == __float_as_uint(b); }
__device__ __forceinline__ bool same_bits(double a, double b) {
    return __double_as_longlong(a) == __double_as_longlong(b);
}
__device__ __forceinline__ bool same_bits(fx2 a, fx2 b) { return same_bits(a.hi, b.hi) && same_bits(a.lo, b.lo); }

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
// inc.cur != 0 (an incremental call): only the nets k_inc_moved stamped are
// re-timed, by the same code.
template <typename R>
__global__ void __launch_bounds__(kRcThreads) k_net_rc(Topo t, State<R> s, const R *__restrict__ x,
                                                       const R *__restrict__ y, double T, R r, R c,
                                                       R d0, int n_small_blocks, Inc inc) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *s.T = T;
        s.gsync[0] = 0u;  // the forward sweep's barrier word (the sweep follows)
    }
    const bool incr = inc.cur != 0;
    if ((int)blockIdx.x < n_small_blocks) {
        const int e = blockIdx.x * kRcThreads + threadIdx.x;
        if (e >= t.n_nets) return;
        if (incr && ldg(&inc.stamp[e]) != inc.cur) return;
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
    if (incr && ldg(&inc.stamp[e]) != inc.cur) return;  // the whole block
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
    s.pred[e] = make_int2(bi, bn);
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
            const A av = AC::add(ldd<COH>(&s.arr[ldg(&t.lv_in_drv[p])]), ldg(&s.tnet[ip]));
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

// ---- one cell per thread (at most kPre inputs: the common case)

// A list entry in registers.  FP32: one 64-bit sort key, the order-
// preserving bits of the cost above the 32-bit ordering key, so that an
// entry compares in one integer comparison; FP64: the pair (cost, key).
__device__ __forceinline__ float from_ord(uint32_t o) {
    return (o & 0x80000000u) ? __uint_as_float(o & 0x7fffffffu) : __uint_as_float(~o);
}

template <typename R>
struct LReg;
template <>
struct LReg<float> {
    using E = uint64_t;
    static __device__ __forceinline__ E make(float d, uint32_t key) {
        return ((uint64_t)ord_bits(d) << 32) | key;
    }
    static __device__ __forceinline__ E none() { return make(r_inf<float>(), kNoneKey); }
    static __device__ __forceinline__ bool before(E a, E b) { return a < b; }
    static __device__ __forceinline__ uint32_t key(E a) { return (uint32_t)a; }
    static __device__ __forceinline__ float cost(E a) { return from_ord((uint32_t)(a >> 32)); }
};
template <>
struct LReg<double> {
    using E = LEnt<double>;
    static __device__ __forceinline__ E make(double d, uint32_t key) { return E{d, key}; }
    static __device__ __forceinline__ E none() { return E{r_inf<double>(), kNoneKey}; }
    static __device__ __forceinline__ bool before(const E &a, const E &b) { return lent_before(a, b); }
    static __device__ __forceinline__ uint32_t key(const E &a) { return a.key; }
    static __device__ __forceinline__ double cost(const E &a) { return a.d; }
};

template <typename R>
__device__ __forceinline__ typename LReg<R>::E lreg_of(float d, int32_t pin) {
    return LReg<R>::make(d, pin < 0 ? kNoneKey : ((1u << 29) | (uint32_t)pin));
}
template <typename R>
__device__ __forceinline__ typename LReg<R>::E lreg_of(double d, int32_t pin) {
    return LReg<R>::make(d, pin < 0 ? kNoneKey : ((1u << 29) | (uint32_t)pin));
}
template <typename R>
__device__ __forceinline__ int32_t lreg_pin(const typename LReg<R>::E &x) {
    const uint32_t k = LReg<R>::key(x);
    return k == kNoneKey ? -1 : (int32_t)(k & kPinMask);
}

// insert x into a sorted list held in registers, keeping its first L entries
// (compare-and-shift from the top); inserting LReg::none() changes nothing
template <typename R, int L>
__device__ __forceinline__ void list_insert(typename LReg<R>::E (&li)[L], const typename LReg<R>::E &x) {
#pragma unroll
    for (int j = L - 1; j >= 0; --j) {
        const bool shift = j > 0 && LReg<R>::before(x, li[j - 1]);
        const bool here = LReg<R>::before(x, li[j]);
        li[j] = shift ? li[j - 1] : (here ? x : li[j]);
    }
}

// list I/O in aligned vectors: a list block is G = L + 1 entries; the entry
// after the L-th is padding (written as a sentinel)
template <int L, bool COH>
__device__ __forceinline__ void list_load(const BEnt<float> *src, uint64_t (&li)[L]) {
    const float4 *v4 = reinterpret_cast<const float4 *>(src);
#pragma unroll
    for (int q = 0; q < list_group(L) / 2; ++q) {
        const float4 v = ldd<COH>(&v4[q]);
        if (2 * q < L) li[2 * q] = lreg_of<float>(v.x, __float_as_int(v.y));
        if (2 * q + 1 < L) li[2 * q + 1] = lreg_of<float>(v.z, __float_as_int(v.w));
    }
}
template <int L, bool COH>
__device__ __forceinline__ void list_load(const BEnt<double> *src, LEnt<double> (&li)[L]) {
#pragma unroll
    for (int j = 0; j < L; ++j) {
        const BEnt<double> v = ldd<COH>(&src[j]);
        li[j] = lreg_of<double>(v.delta, v.pin);
    }
}
template <int L>
__device__ __forceinline__ void list_put(BEnt<float> *dst, const uint64_t (&li)[L]) {
    float4 *v4 = reinterpret_cast<float4 *>(dst);
#pragma unroll
    for (int q = 0; q < list_group(L) / 2; ++q) {
        const uint64_t x = 2 * q < L ? li[2 * q] : LReg<float>::none();
        const uint64_t y = 2 * q + 1 < L ? li[2 * q + 1] : LReg<float>::none();
        v4[q] = make_float4(LReg<float>::cost(x), __int_as_float(lreg_pin<float>(x)), LReg<float>::cost(y),
                            __int_as_float(lreg_pin<float>(y)));
    }
}
template <int L>
__device__ __forceinline__ void list_put(BEnt<double> *dst, const LEnt<double> (&li)[L]) {
#pragma unroll
    for (int j = 0; j < L; ++j) dst[j] = BEnt<double>{li[j].d, lreg_pin<double>(li[j])};
}

// Lists moved by a whole warp.  With per-thread vector I/O (list_load,
// list_put) every load or store instruction of a warp touches 32 lists, one
// 16-byte piece of each: 32 L2 requests for 512 bytes, each sector fetched
// twice.  Here each instruction moves 512 / B whole lists of B bytes, the
// pieces of one list on consecutive lanes (B >= 128: four requests of a full
// 128-byte line), and the pieces pass between the lanes through a per-warp
// staging area in shared memory (32 * C pieces).  The lists and their bits
// are those of list_load / list_put.
template <typename R, int L>
struct WarpList {
    static constexpr int G = list_group(L);
    static constexpr int B = G * (int)sizeof(BEnt<R>);  // bytes of a list block
    static constexpr int C = B / 16;                     // 16-byte pieces of a list
    static constexpr int LPI = 32 / C;                   // lists per instruction
    static constexpr int SPREAD = C >= 8 ? 1 : 8 / C;
    static_assert(B % 16 == 0 && C >= 2 && C <= 32, "list block of 2 to 32 pieces");
    // staging slot of piece q of lane i's list: the pieces of a list are
    // rotated within its C slots so that the eight lanes of a quarter warp
    // reading piece q of their own lists meet eight different 16-byte bank
    // groups (the writes of an instruction cover consecutive slots)
    static __device__ __forceinline__ int slot(int i, int q) { return i * C + (q + i / SPREAD) % C; }
};

// the 16-byte piece q of a list in registers, as list_put stores it
template <int L>
__device__ __forceinline__ float4 list_piece(const uint64_t (&li)[L], int q) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int r = 0; r < list_group(L) / 2; ++r) {
        if (r == q) {
            const uint64_t x = 2 * r < L ? li[2 * r] : LReg<float>::none();
            const uint64_t y = 2 * r + 1 < L ? li[2 * r + 1] : LReg<float>::none();
            v = make_float4(LReg<float>::cost(x), __int_as_float(lreg_pin<float>(x)), LReg<float>::cost(y),
                            __int_as_float(lreg_pin<float>(y)));
        }
    }
    return v;
}
template <int L>
__device__ __forceinline__ float4 list_piece(const LEnt<double> (&li)[L], int q) {
    double d = r_inf<double>();
    int32_t pin = -1;
#pragma unroll
    for (int r = 0; r < L; ++r) {
        if (r == q) {
            d = li[r].d;
            pin = lreg_pin<double>(li[r]);
        }
    }
    const double2 v = make_double2(d, __longlong_as_double((long long)(uint32_t)pin));
    return *reinterpret_cast<const float4 *>(&v);
}
// piece q of a list into registers, as list_load reads it
template <int L>
__device__ __forceinline__ void list_unpiece(float4 v, int q, uint64_t (&li)[L]) {
#pragma unroll
    for (int r = 0; r < list_group(L) / 2; ++r) {
        if (r == q) {
            if (2 * r < L) li[2 * r] = lreg_of<float>(v.x, __float_as_int(v.y));
            if (2 * r + 1 < L) li[2 * r + 1] = lreg_of<float>(v.z, __float_as_int(v.w));
        }
    }
}
template <int L>
__device__ __forceinline__ void list_unpiece(float4 v, int q, LEnt<double> (&li)[L]) {
    const double2 w = *reinterpret_cast<const double2 *>(&v);
#pragma unroll
    for (int r = 0; r < L; ++r)
        if (r == q) li[r] = lreg_of<double>(w.x, (int32_t)(__double_as_longlong(w.y) & 0xffffffffll));
}

// Every lane of the warp calls these.  src / dst: the net whose list the
// lane reads / writes (< 0: none; a lane without a list to read gets
// sentinels).  The staging area is free again when they return.  The loads
// go from L2 to the staging area as asynchronous copies (cp.async.cg: read
// from L2 like ld.global.cg, so COH makes no difference here, and no
// registers held while they are in flight); the staging area is addressed in
// the shared window (32-bit addresses).
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
// the lane index read afresh at each call, so that the compiler recomputes
// the staging offsets (a few integer operations) instead of holding them in
// registers across the whole sweep
__device__ __forceinline__ int lane_now() {
    int l;
    asm volatile("mov.u32 %0, %%laneid;" : "=r"(l));
    return l;
}
__device__ __forceinline__ float4 lds16(unsigned a) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
    return v;
}
__device__ __forceinline__ void sts16(unsigned a, float4 v) {
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}
// the copies of the lists src (per lane) into the staging area, not waited for
template <typename R, int L>
__device__ __forceinline__ void warp_list_issue(const BEnt<R> *blist, int src, unsigned st0) {
    using W = WarpList<R, L>;
    const int lane = lane_now();
#pragma unroll
    for (int t = 0; t < W::C; ++t) {
        const int i = t * W::LPI + lane / W::C, q = lane % W::C;
        const int n = __shfl_sync(0xffffffffu, src, i);
        if (n >= 0) {
            const float4 *g = reinterpret_cast<const float4 *>(blist + (size_t)n * W::G) + q;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(st0 + 16u * (unsigned)W::slot(i, q)),
                         "l"(g)
                         : "memory");
        }
    }
}
// every lane unpacks its list from the staging area at st0 (after the
// copies were waited for); a lane without a list (has false) takes
// sentinels (a select per entry, not a branch around the unpacking)
template <typename R, int L>
__device__ __forceinline__ void warp_list_take(unsigned st0, bool has, typename LReg<R>::E (&li)[L]) {
    using W = WarpList<R, L>;
    const int lane = lane_now();
#pragma unroll
    for (int q = 0; q < W::C; ++q) list_unpiece<L>(lds16(st0 + 16u * (unsigned)W::slot(lane, q)), q, li);
#pragma unroll
    for (int j = 0; j < L; ++j) li[j] = has ? li[j] : LReg<R>::none();
}
template <typename R, int L, bool COH>
__device__ __forceinline__ void warp_list_load(const BEnt<R> *blist, int src, float4 *stage,
                                               typename LReg<R>::E (&li)[L]) {
    const unsigned st0 = smem_u32(stage);
    warp_list_issue<R, L>(blist, src, st0);
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncwarp();
    warp_list_take<R, L>(st0, src >= 0, li);
    __syncwarp();
}

// Whether a warp fetches the lists of all of a cell's inputs at once (one
// staging area per input slot, kPre of them), issued right after the loads
// of the inputs' arrivals, so that the worst input's list needs no load of
// its own after the argmax: where kPre staging areas of a 256-thread block
// fit in shared memory (lists of at most 128 bytes). Issued before the
// arrival loads, the copies delay them and the sweep gets slower.
template <typename R, int L>
__host__ __device__ constexpr bool all_lists() {
    return L > 0 && (size_t)list_group(L) * sizeof(BEnt<R>) <= 128;
}
template <typename R, int L>
__device__ __forceinline__ void warp_list_put(BEnt<R> *blist, int dst, float4 *stage,
                                              const typename LReg<R>::E (&li)[L]) {
    using W = WarpList<R, L>;
    const int lane = lane_now();
    const unsigned st0 = smem_u32(stage);
#pragma unroll
    for (int q = 0; q < W::C; ++q) sts16(st0 + 16u * (unsigned)W::slot(lane, q), list_piece<L>(li, q));
    __syncwarp();
#pragma unroll
    for (int t = 0; t < W::C; ++t) {
        const int i = t * W::LPI + lane / W::C, q = lane % W::C;
        const int n = __shfl_sync(0xffffffffu, dst, i);
        const float4 v = lds16(st0 + 16u * (unsigned)W::slot(i, q));
        if (n >= 0) reinterpret_cast<float4 *>(blist + (size_t)n * W::G)[q] = v;
    }
    __syncwarp();
}

// bytes of the staging area a block of `threads` threads needs for lists of L
// (kPre areas a warp where all_lists<R, L>() holds)
template <typename R>
__host__ __device__ constexpr size_t warp_list_smem(int L, int threads) {
    return L == 0 ? 0
                  : (size_t)threads * (size_t)list_group(L) * sizeof(BEnt<R>) *
                        ((size_t)list_group(L) * sizeof(BEnt<R>) <= 128 ? kPre : 1);
}

// whether the stored list at dst holds, bit for bit, what list_put(dst, li)
// would write
template <int L>
__device__ __forceinline__ bool list_same(const BEnt<float> *dst, const uint64_t (&li)[L]) {
    const float4 *v4 = reinterpret_cast<const float4 *>(dst);
    bool same = true;
#pragma unroll
    for (int q = 0; q < list_group(L) / 2; ++q) {
        const uint64_t x = 2 * q < L ? li[2 * q] : LReg<float>::none();
        const uint64_t y = 2 * q + 1 < L ? li[2 * q + 1] : LReg<float>::none();
        const float4 o = __ldcg(&v4[q]);
        same = same && same_bits(o.x, LReg<float>::cost(x)) && __float_as_int(o.y) == lreg_pin<float>(x) &&
               same_bits(o.z, LReg<float>::cost(y)) && __float_as_int(o.w) == lreg_pin<float>(y);
    }
    return same;
}
template <int L>
__device__ __forceinline__ bool list_same(const BEnt<double> *dst, const LEnt<double> (&li)[L]) {
    bool same = true;
#pragma unroll
    for (int j = 0; j < L; ++j) {
        const BEnt<double> o = ldcg(&dst[j]);
        same = same && same_bits(o.delta, li[j].d) && o.pin == lreg_pin<double>(li[j]);
    }
    return same;
}

// One cell for one thread: cell k (k < 0: none), its inputs when it has at
// most kPre, and, once loaded (vals), the values that stay fixed during the
// sweep (the cell delay, the inputs' Elmore delays) and the arrival and chain
// length of drivers two or more levels down (bit u of old).
template <typename R>
struct CellPre {
    using A = typename Acc<R>::T;
    int k, a, b, e, o;
    int ip[kPre], in[kPre], dv[kPre];
    unsigned fl, old;
    bool vals;
    R dcell;
    R tv[kPre];
    A ad[kPre];
    int pl[kPre];
};

// topology of cell k: the cell record and its input slots, one round of loads
template <typename R>
__device__ __forceinline__ void cell_topo(const Topo &t, int k, CellPre<R> &c) {
    c.k = k;
    c.a = c.b = 0;
    c.fl = c.old = 0u;
    c.vals = false;
    if (k < 0) return;
    const int4 r = ldg(&t.lv_rec[k]);
    int4 sl[kPre];
#pragma unroll
    for (int u = 0; u < kPre; ++u) sl[u] = ldg(&t.lv_slot[(size_t)k * kPre + u]);
    c.e = r.x;
    c.o = r.y;
    c.a = r.w;
    c.b = r.w + r.z;
    const int nin = r.z;
    if (nin > kPre) return;
#pragma unroll
    for (int u = 0; u < kPre; ++u) {
        if (u < nin) {
            c.ip[u] = sl[u].x;
            c.in[u] = sl[u].y;
            c.dv[u] = sl[u].z;
            c.fl |= (unsigned)sl[u].w << (8 * u);
        }
    }
}

// the values of cell c that are already final before the barrier that opens
// its level (single launch): one round of loads
template <typename R>
__device__ __forceinline__ void cell_vals(const State<R> &s, CellPre<R> &c) {
    if (c.k < 0) return;
    const int nin = c.b - c.a;
    if (nin > kPre) return;
    c.dcell = ldg(&s.dnet[c.e]);
#pragma unroll
    for (int u = 0; u < kPre; ++u) {
        if (u < nin) {
            c.tv[u] = ldg(&s.tnet[c.ip[u]]);
            if (!((c.fl >> (8 * u)) & kInPrev)) {
                c.ad[u] = ldcg(&s.arr[c.dv[u]]);
                c.pl[u] = ldcg(&s.plen[c.in[u]]);
                c.old |= 1u << u;
            }
        }
    }
    c.vals = true;
}

// Arrival of one cell (Section II-B: max over its inputs of the driver's
// arrival plus the Elmore delay, plus the cell delay) and, when L > 0, its
// sidetrack list.  The input pins' arrivals are not stored: nothing in a
// timing iteration reads them, and k_in_arr forms them, with the same
// addition, when sta_get_timing asks.  COH: the drivers' values were written by other blocks of
// the same launch.  CMP: returns whether the cell's output arrival, worst
// input, chain length or list differs, bit for bit, from what was stored
// before (a cell of more than kPre inputs always counts as changed).

// WARP: every lane of the warp calls it (a lane without a cell passes
// k < 0) and the lists move as whole lists (warp_list_load / _put, staging
// area `stage`); else the lane alone, with per-thread list I/O.
template <typename R, int L, bool COH, bool CMP = false, bool WARP = false>
__device__ __forceinline__ bool fwd_cell(const Topo &t, State<R> &s, const CellPre<R> &c,
                                         float4 *stage = nullptr) {
    static_assert(!(CMP && WARP), "the comparing form runs lane by lane");
    using AC = Acc<R>;
    using A = typename AC::T;
    using LR = LReg<R>;
    bool act = c.k >= 0;
    if constexpr (!WARP) {
        if (!act) return false;
    }
    const int nin = c.b - c.a;
    if (act && nin > kPre) {
        fwd_cell_wide<R, L, COH>(t, s, c.k, c.a, c.b);
        if constexpr (!WARP) return true;
        act = false;  // its list is built; the lane only joins the warp's list moves
    }
    // every load first, then the arithmetic, then the stores
    int bi = -1, bn = -1, bl = 0, bu = 0;
    A best = AC::ninf();
    A av[kPre];
    bool chg = false;
    [[maybe_unused]] unsigned lst0 = 0;
    R dcell = R(0);
    R tv[kPre];
    int pl[kPre];
    if (act) {
        dcell = c.vals ? c.dcell : ldg(&s.dnet[c.e]);
#pragma unroll
        for (int u = 0; u < kPre; ++u) {
            if (u < nin) {
                tv[u] = c.vals ? c.tv[u] : ldg(&s.tnet[c.ip[u]]);
                if ((c.old >> u) & 1u) {
                    av[u] = c.ad[u];
                    pl[u] = c.pl[u];
                } else {
                    av[u] = ldd<COH>(&s.arr[c.dv[u]]);
                    pl[u] = ldd<COH>(&s.plen[c.in[u]]);
                }
            }
        }
    }
    if constexpr (WARP && all_lists<R, L>()) {
        // the lists of every input from a combinational cell, into one
        // staging area per input slot, right after the inputs' arrivals
        constexpr unsigned kArea = 32u * WarpList<R, L>::C * 16u;
        lst0 = smem_u32(stage);
#pragma unroll
        for (int u = 0; u < kPre; ++u) {
            const bool lu = act && u < nin && ((c.fl >> (8 * u)) & kInComb);
            warp_list_issue<R, L>(s.blist, lu ? c.in[u] : -1, lst0 + (unsigned)u * kArea);
        }
    }
    if (act) {
        // inputs ascending by pin: strict > keeps the lowest pin on ties (and
        // the first input if arrivals are not comparable)
#pragma unroll
        for (int u = 0; u < kPre; ++u) {
            if (u < nin) {
                av[u] = AC::add(av[u], tv[u]);
                if (bi < 0 || AC::gt(av[u], best)) {
                    best = av[u];
                    bi = c.ip[u];
                    bn = c.in[u];
                    bl = pl[u];
                    bu = u;
                }
            }
        }
        if constexpr (CMP) {
            const int2 op = ldcg(&s.pred[c.e]);
            chg = !same_bits(ldcg(&s.arr[c.o]), AC::add(best, dcell)) || op.x != bi || op.y != bn ||
                  ldcg(&s.plen[c.e]) != bl + 2;
        }
        s.arr[c.o] = AC::add(best, dcell);
        s.pred[c.e] = make_int2(bi, bn);
        s.plen[c.e] = bl + 2;
    }
    if constexpr (L > 0) {
        constexpr int G = list_group(L);
        typename LR::E li[L];
        const bool from = act && nin > 0 && ((c.fl >> (8 * bu)) & kInComb);
        if constexpr (WARP && all_lists<R, L>()) {
            // the worst input's list from that input's staging area
            constexpr unsigned kArea = 32u * WarpList<R, L>::C * 16u;
            asm volatile("cp.async.wait_all;" ::: "memory");
            __syncwarp();
            warp_list_take<R, L>(lst0 + (unsigned)bu * kArea, from, li);
            __syncwarp();
        } else if constexpr (WARP) {
            warp_list_load<R, L, COH>(s.blist, from ? bn : -1, stage, li);
        } else if (from) {
            list_load<L, COH>(s.blist + (size_t)bn * G, li);
        } else {
#pragma unroll
            for (int j = 0; j < L; ++j) li[j] = LR::none();
        }
        if (act) {
            // the own deviations: every input but the worst, kPre - 1 slots
            // (absent ones as no-op sentinels, so that the threads of a warp
            // do not diverge), inserted in input order
            typename LR::E prev = LR::none();
#pragma unroll
            for (int u = 0; u < kPre; ++u) {
                const uint32_t key = ((c.ip[u] < bi ? 0u : 2u) << 29) | (uint32_t)c.ip[u];
                const typename LR::E e = u < nin && u != bu ? LR::make(AC::diff(best, av[u]), key) : LR::none();
                // slot u - 1 takes input u - 1 below the worst input, input u from it on
                if (u > 0) list_insert<R, L>(li, u - 1 < bu ? prev : e);
                prev = e;
            }
        }
        if constexpr (CMP) {
            int m = 0;
#pragma unroll
            for (int j = 0; j < L; ++j) m += LR::key(li[j]) == kNoneKey ? 0 : 1;
            chg = chg || ldcg(&s.bcnt[c.e]) != m || !list_same<L>(s.blist + (size_t)c.e * G, li);
        }
        if constexpr (WARP) warp_list_put<R, L>(s.blist, act ? c.e : -1, stage, li);
        else list_put<L>(s.blist + (size_t)c.e * G, li);
        if (act) {
            int m = 0;
#pragma unroll
            for (int j = 0; j < L; ++j) m += LR::key(li[j]) == kNoneKey ? 0 : 1;
            s.bcnt[c.e] = m;
        }
    }
    return chg;
}

// One launch per level (captured in a CUDA graph): a thread per cell.
template <typename R, int L>
__global__ void __launch_bounds__(kLvThreads) k_fwd_level(Topo t, State<R> s, int lo, int hi) {
    pdl_trigger();
    const int k = lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= hi) return;
    CellPre<R> c;
    cell_topo(t, k, c);
    pdl_wait();  // the timing loads read what earlier launches wrote
    fwd_cell<R, L, false>(t, s, c);
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

// Single-launch sweeps: one block per SM (kFwdThreads / kBwdThreads threads),
// a level's work cut into warp-sized chunks, chunk j on block j mod gridDim
// so that a level is spread over every SM.
constexpr int kFwdThreads = 256;
// (the backward sweep: 28 warps a block, which its 68-72 registers allow,
// so that fewer SMs take a level's tasks in one round)
constexpr int kBwdThreads = 896;

// The whole forward sweep in one cooperative launch: levels in order, a
// thread per cell, a grid-wide barrier between levels.  A thread carries its
// first cell of the next two levels: between its arrival at the barrier that
// closes level l and the wait, it loads, in one round, the final values of
// its level l + 1 cell (cell delay, Elmore delays, drivers two or more
// levels down) and the topology of its level l + 2 cell, so that after the
// barrier only the values level l wrote are left to load.  from (if not
// NULL): the first level to evaluate, in device memory (an incremental
// propagation hands over the levels after the one where its changes
// saturated; past the last level: nothing to do); else level 1.
template <typename R, int L>
__global__ void __launch_bounds__(kFwdThreads, 1) k_fwd_sweep(Topo t, State<R> s, GridSync gs,
                                                               const int *from) {
    const int lane = threadIdx.x & 31;
    const int w0 = blockIdx.x + (threadIdx.x >> 5) * gridDim.x;  // first chunk of this warp
    const int wstride = (blockDim.x >> 5) * gridDim.x;
    auto cell_of = [&](int l, int chunk) {
        if (l > t.depth) return -1;
        const int k = ldg(&t.lvl_ptr[l - 1]) + chunk * 32 + lane;
        return k < ldg(&t.lvl_ptr[l]) ? k : -1;
    };
    // staging area of this warp's list moves (warp_list_smem bytes a block)
    extern __shared__ float4 lstage[];
    float4 *stage = lstage + (size_t)(threadIdx.x >> 5) * 32 * (L > 0 ? WarpList<R, L>::C : 0) *
                                 (all_lists<R, L>() ? kPre : 1);
    const int l0 = from ? max(ldcg(from), 1) : 1;
    if (l0 > t.depth) return;
    CellPre<R> cur, nxt;
    cell_topo(t, cell_of(l0, w0), cur);
    cell_topo(t, cell_of(l0 + 1, w0), nxt);
    for (int l = l0; l <= t.depth; ++l) {
        const int nch = div_up_dev(ldg(&t.lvl_ptr[l]) - ldg(&t.lvl_ptr[l - 1]), 32);
        if (w0 < nch) {  // the same in every lane of the warp
            fwd_cell<R, L, true, false, true>(t, s, cur, stage);
            for (int ch = w0 + wstride; ch < nch; ch += wstride) {
                CellPre<R> c;
                cell_topo(t, cell_of(l, ch), c);
                fwd_cell<R, L, true, false, true>(t, s, c, stage);
            }
        }
        if (l == t.depth) break;
        grid_arrive(gs);
        cur = nxt;
        cell_vals(s, cur);                // drivers below level l are final
        cell_topo(t, cell_of(l + 2, w0), nxt);
        if (!grid_wait(gs, (unsigned)(l - l0 + 1) * gridDim.x)) return;
    }
}

// ----------------------------------------------------- incremental ---
//
// sta_propagate_incremental re-times only what the moved cells reach, with
// the code of the full propagation, so that its results are bit for bit
// those of a full one:
//   k_inc_moved      cells whose position differs (bit for bit) from the
//                    last propagation: record the new one, stamp their nets
//                    (their delays may change) and widen the call's level
//                    span [lo, hi] to the levels those nets reach
//   k_net_rc         (incremental mode) re-times the stamped nets
//   k_fwd_sweep_inc  levels lo .. hi: a cell is re-evaluated when its net or
//                    an input's net is stamped; a re-evaluated cell whose
//                    outputs changed stamps its net and raises hi to the
//                    deepest level that net reaches; once the changes of a
//                    level saturate, it stops and k_fwd_sweep evaluates every
//                    cell of the levels after

// Level span of each net: the level of its driving cell when that is
// combinational (its delay depends on the net's load), and the levels of
// the combinational cells it feeds.  (INT_MAX, 0) when there are none.
__global__ void k_inc_span(Topo t, int2 *span) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= t.n_nets) return;
    const int d = ldg(&t.net_level[e]);
    int lo = d >= 1 ? d : INT_MAX, hi = d;
    for (int p = ldg(&t.net_ptr[e]) + 1; p < ldg(&t.net_ptr[e + 1]); ++p) {
        const int on = ldg(&t.sink_onet[p]);
        if (on < 0) continue;
        const int l = ldg(&t.net_level[on]);
        lo = min(lo, l);
        hi = max(hi, l);
    }
    span[e] = make_int2(lo, hi);
}

// Level span of each cell: the spans of the nets of its pins, combined.
__global__ void k_inc_cspan(Topo t, const int2 *span, int2 *cspan) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= t.n_cells) return;
    int lo = INT_MAX, hi = 0;
    for (int q = ldg(&t.cp_ptr[c]); q < ldg(&t.cp_ptr[c + 1]); ++q) {
        const int2 sp = ldg(&span[ldg(&t.pin_net[ldg(&t.cp[q])])]);
        lo = min(lo, sp.x);
        hi = max(hi, sp.y);
    }
    cspan[c] = make_int2(lo, hi);
}

__global__ void k_inc_reset(Inc inc) {
    if (threadIdx.x < 3) inc.cnt[threadIdx.x] = 0ull;
    if (threadIdx.x == 0) {
        inc.lohi[0] = INT_MAX;
        inc.lohi[1] = 0;
        inc.lohi[2] = INT_MAX;
    }
}

// Widen the call's level span (checked first: the atomics fire only while
// the span grows).
__device__ __forceinline__ void inc_widen(const Inc &inc, int lo, int hi) {
    if (lo < ldcg(&inc.lohi[0])) atomicMin(&inc.lohi[0], lo);
    if (hi > ldcg(&inc.lohi[1])) atomicMax(&inc.lohi[1], hi);
}

template <typename R>
__global__ void k_inc_moved(Topo t, const R *__restrict__ x, const R *__restrict__ y, R *xp, R *yp, Inc inc) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    bool mv = false;
    if (c < t.n_cells) {
        const R xv = ldg(&x[c]), yv = ldg(&y[c]);
        mv = !same_bits(xv, xp[c]) || !same_bits(yv, yp[c]);
        if (mv) {
            xp[c] = xv;
            yp[c] = yv;
            for (int q = ldg(&t.cp_ptr[c]); q < ldg(&t.cp_ptr[c + 1]); ++q)
                inc.stamp[ldg(&t.pin_net[ldg(&t.cp[q])])] = inc.cur;
            const int2 sp = ldg(&inc.cspan[c]);
            inc_widen(inc, sp.x, sp.y);
        }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, mv);
    if ((threadIdx.x & 31) == 0 && bal) atomicAdd(&inc.cnt[0], (unsigned long long)__popc(bal));
}

// Stamps of cell c that are final before the barrier opening its level: its
// own net (its delay) and the nets of inputs driven two or more levels down.
// (Bitwise or, not ||: the loads are issued together.)
template <typename R>
__device__ __forceinline__ bool inc_dirty_old(const Inc &inc, const CellPre<R> &c) {
    if (c.k < 0) return false;
    bool d = ldcg(&inc.stamp[c.e]) == inc.cur;
    if (c.b - c.a <= kPre) {
#pragma unroll
        for (int u = 0; u < kPre; ++u)
            if (u < c.b - c.a && !((c.fl >> (8 * u)) & kInPrev)) d |= ldcg(&inc.stamp[c.in[u]]) == inc.cur;
    }
    return d;
}

// One cell of the incremental sweep.  After the barrier, in one round: the
// stamps of the inputs driven by the level below and (whether or not they
// show a change) those drivers' arrivals and chain lengths, the only values
// cell_vals left out.  If a stamp is set, the cell's full evaluation, which
// then loads nothing but the worst input's list.  A wide cell (more than
// kPre inputs) checks every input's stamp first.
template <typename R, int L>
__device__ __forceinline__ void inc_cell(const Topo &t, State<R> &s, const Inc &inc, CellPre<R> &c, bool d,
                                         int &hi, unsigned &n_eval, unsigned &n_chg) {
    if (c.k < 0) return;
    const int nin = c.b - c.a;
    if (nin > kPre) {
        for (int p = c.a; p < c.b && !d; ++p) d = ldcg(&inc.stamp[ldg(&t.lv_in_net[p])]) == inc.cur;
    } else {
#pragma unroll
        for (int u = 0; u < kPre; ++u) {
            if (u < nin && ((c.fl >> (8 * u)) & kInPrev)) {
                d |= ldcg(&inc.stamp[c.in[u]]) == inc.cur;
                c.ad[u] = ldcg(&s.arr[c.dv[u]]);
                c.pl[u] = ldcg(&s.plen[c.in[u]]);
                c.old |= 1u << u;
            }
        }
    }
    if (!d) return;
    ++n_eval;
    if (fwd_cell<R, L, true, true>(t, s, c)) {
        inc.stamp[c.e] = inc.cur;
        hi = max(hi, ldg(&inc.span[c.e]).y);
        ++n_chg;
    }
}

// A level whose changed cells exceed 1/kIncSaturate of the next level's
// cells ends the selective part of the sweep: k_fwd_sweep, launched after
// it, evaluates every cell of the following levels, without stamps or
// comparisons.  The changes of a few moved cells spread through the
// sidetrack lists to most of the cells downstream, and there the checks only
// lengthen each level.
constexpr int kIncSaturate = 16;

// The incremental forward sweep: one cooperative launch over levels lo .. hi
// of this call (hi grows as changes reach deeper cells), the layout of
// k_fwd_sweep (a thread per cell, chunk j of a level on block j mod
// gridDim; in the barrier window, the next level's values and stamps that
// are already final and the topology of the level after).  When the
// changes saturate after level l, it records l + 1 in lohi[2] and stops.
// Every block reads the same lo; a block may read a larger hi than another
// after a barrier, but only once some block has continued past it, so all
// blocks leave the loop after the same level.
template <typename R, int L>
__global__ void __launch_bounds__(kFwdThreads, 1) k_fwd_sweep_inc(Topo t, State<R> s, GridSync gs, Inc inc) {
    __shared__ int blk_hi;
    const int lane = threadIdx.x & 31;
    const int w0 = blockIdx.x + (threadIdx.x >> 5) * gridDim.x;
    const int wstride = (blockDim.x >> 5) * gridDim.x;
    auto cell_of = [&](int l, int chunk) {
        if (l > t.depth) return -1;
        const int k = ldg(&t.lvl_ptr[l - 1]) + chunk * 32 + lane;
        return k < ldg(&t.lvl_ptr[l]) ? k : -1;
    };
    __shared__ int blk_chg;
    const int lo = ldcg(&inc.lohi[0]);
    int hi = min(ldcg(&inc.lohi[1]), t.depth);
    unsigned n_eval = 0, n_chg = 0, nbar = 0;
    if (threadIdx.x == 0) blk_hi = blk_chg = 0;
    __syncthreads();
    CellPre<R> cur, nxt;
    bool cur_d = false;
    if (lo <= hi) {
        cell_topo(t, cell_of(lo, w0), cur);
        cell_topo(t, cell_of(lo + 1, w0), nxt);
        cell_vals(s, cur);
        cur_d = inc_dirty_old(inc, cur);
    }
    for (int l = lo; l <= hi; ++l) {
        const int nch = div_up_dev(ldg(&t.lvl_ptr[l]) - ldg(&t.lvl_ptr[l - 1]), 32);
        int h = 0;
        const unsigned c0 = n_chg;
        if (w0 < nch) {
            inc_cell<R, L>(t, s, inc, cur, cur_d, h, n_eval, n_chg);
            for (int ch = w0 + wstride; ch < nch; ch += wstride) {
                CellPre<R> c;
                cell_topo(t, cell_of(l, ch), c);
                cell_vals(s, c);
                inc_cell<R, L>(t, s, inc, c, inc_dirty_old(inc, c), h, n_eval, n_chg);
            }
        }
        h = __reduce_max_sync(0xffffffffu, h);
        const unsigned dc = __reduce_add_sync(0xffffffffu, n_chg - c0);
        if (lane == 0 && h > 0) atomicMax(&blk_hi, h);
        if (lane == 0 && dc > 0) atomicAdd(&blk_chg, (int)dc);
        __syncthreads();
        if (threadIdx.x == 0) {
            // ordered before the block's release arrival below by its block barrier
            if (blk_hi > 0) atomicMax(&inc.lohi[1], blk_hi);
            if (blk_chg > 0) atomicAdd(&inc.lvchg[l], blk_chg);
            blk_hi = blk_chg = 0;
        }
        if (l == t.depth) break;
        grid_arrive(gs);
        ++nbar;
        cur = nxt;
        cell_vals(s, cur);                // values and stamps below level l are final
        cur_d = inc_dirty_old(inc, cur);
        cell_topo(t, cell_of(l + 2, w0), nxt);
        if (!grid_wait(gs, nbar * gridDim.x)) return;
        // the same counts in every block: level l's are final after the barrier
        const int next = ldg(&t.lvl_ptr[l + 1]) - ldg(&t.lvl_ptr[l]);
        if ((long long)ldcg(&inc.lvchg[l]) * kIncSaturate > next) {
            if (blockIdx.x == 0 && threadIdx.x == 0) inc.lohi[2] = l + 1;
            break;
        }
        hi = min(ldcg(&inc.lohi[1]), t.depth);
    }
    n_eval = __reduce_add_sync(0xffffffffu, n_eval);
    n_chg = __reduce_add_sync(0xffffffffu, n_chg);
    if (lane == 0 && n_eval) {
        atomicAdd(&inc.cnt[1], (unsigned long long)n_eval);
        if (n_chg) atomicAdd(&inc.cnt[2], (unsigned long long)n_chg);
    }
}

// ----------------------------------------------------------- backward ---

template <typename T>
__device__ __forceinline__ T shfl_x(T v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ fx2 shfl_x(fx2 v, int o) {
    return fx2{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}

// A net's required time travels as an order-preserving 64-bit key, so that
// the pieces of a large net combine with one integer atomicMin (exact, and
// independent of their order): FP32 pairs as (hi bits, lo bits), which
// orders them as Acc<float>::lt does; FP64 as its own bits.  All ones stands
// for +inf (a net with no sink).
constexpr unsigned long long kKeyNone = ~0ull;
__device__ __forceinline__ unsigned long long acc_key(fx2 v) {
    return ((unsigned long long)ord_bits(v.hi) << 32) | ord_bits(v.lo);
}
__device__ __forceinline__ unsigned long long acc_key(double v) { return ord_bits(v); }
__device__ __forceinline__ double from_ord64(uint64_t o) {
    return (o & 0x8000000000000000ull) ? __longlong_as_double((long long)(o & 0x7fffffffffffffffull))
                                       : __longlong_as_double((long long)~o);
}
template <typename R>
__device__ __forceinline__ typename Acc<R>::T acc_unkey(unsigned long long k);
template <>
__device__ __forceinline__ fx2 acc_unkey<float>(unsigned long long k) {
    if (k == kKeyNone) return Acc<float>::pinf();
    return fx2{from_ord((uint32_t)(k >> 32)), from_ord((uint32_t)k)};
}
template <>
__device__ __forceinline__ double acc_unkey<double>(unsigned long long k) {
    if (k == kKeyNone) return Acc<double>::pinf();
    return from_ord64(k);
}

// One lane's share of a backward task (task w, lane): the net's driver pin a
// (a < 0: none) and net e, whether the net is split into pieces, the lane's
// sinks (pin -1: none) with their kind and the net their cell drives, and,
// once loaded (vals), the values that stay fixed during the sweep and, for
// sinks whose cell is two or more levels up (bit j of old), that cell's
// required time.
template <typename R>
struct SinkPre {
    using A = typename Acc<R>::T;
    int a, e, gl;  // gl: lanes of the net (small nets)
    bool split, vals;
    int p[kBwPerLane], kd[kBwPerLane], sn[kBwPerLane];
    unsigned old;
    R tp[kBwPerLane], dn[kBwPerLane];
    A rq[kBwPerLane];
};

// topology: one round of loads (task < 0: none)
template <typename R>
__device__ __forceinline__ void sink_topo(const Topo &t, int task, int lane, SinkPre<R> &c) {
    c.vals = c.split = false;
    c.old = 0u;
    c.a = -1;
    c.gl = 1;
#pragma unroll
    for (int j = 0; j < kBwPerLane; ++j) c.p[j] = -1;
    if (task < 0) return;
    const int2 d = ldg(&t.bw_drv[(size_t)task * 32 + lane]);
    c.a = d.x < 0 ? -1 : (d.x & kBwPinMask);
    c.split = d.x >= 0 && (d.x & kBwSplit);
    c.gl = d.x >= 0 && (d.x & kBwG4) ? 4 : d.x >= 0 && (d.x & kBwG2) ? 2 : 1;
    c.e = d.y;
#pragma unroll
    for (int j = 0; j < kBwPerLane; ++j) {
        const int4 q = ldg(&t.bw_slot[((size_t)task * 32 + lane) * kBwPerLane + j]);
        c.p[j] = q.x;
        c.kd[j] = q.y;
        c.sn[j] = q.z;
    }
}

// the values that are final before the barrier that opens the net's level
// (single launch): one round of loads
template <typename R>
__device__ __forceinline__ void sink_vals(const State<R> &s, SinkPre<R> &c) {
    if (c.a < 0) return;
#pragma unroll
    for (int j = 0; j < kBwPerLane; ++j) {
        if (c.p[j] < 0) continue;
        c.tp[j] = ldg(&s.tnet[c.p[j]]);
        if ((c.kd[j] & kKindMask) != PK_ENDPOINT) {
            c.dn[j] = ldg(&s.dnet[c.sn[j]]);
            if (!(c.kd[j] & kKindPrev)) {
                c.rq[j] = acc_unkey<R>(ldcg(&s.reqkey[c.sn[j]]));
                c.old |= 1u << j;
            }
        }
    }
    c.vals = true;
}

// The net's required time (Section II-B: min over its sinks of the sink's
// required time minus its Elmore delay; a sink's required time is its
// cell's output required time minus the cell delay, or T at an endpoint)
// into reqkey (stored, or atomicMin for the pieces of a split net).  Only
// the nets' required times are stored: those of pins, and slacks, are
// formed on request (k_pin_req, k_pin_slack), the endpoints' by k_ep_wns.
// Required times need no arrival.  PIECE: the warp holds one piece (min over 32 lanes), else small
// nets on aligned groups of 1, 2 or 4 lanes (min over the group).  Every lane of the warp
// calls this.  COH: required times of sink cells were written by other
// blocks of the same launch.
template <typename R, bool COH>
__device__ __forceinline__ void bwd_net(State<R> &s, const SinkPre<R> &c, int lane, bool piece) {
    using AC = Acc<R>;
    using A = typename AC::T;
    A m = AC::pinf();
    if (c.a >= 0) {
        A rq[kBwPerLane];
        R tp[kBwPerLane];
#pragma unroll
        for (int j = 0; j < kBwPerLane; ++j) {  // loads
            if (c.p[j] < 0) continue;
            tp[j] = c.vals ? c.tp[j] : ldg(&s.tnet[c.p[j]]);
            if ((c.kd[j] & kKindMask) == PK_ENDPOINT) {
                rq[j] = acc_from_double<R>(*s.T);  // arrival and slack: k_ep_wns
            } else {
                rq[j] = (c.old >> j) & 1u ? c.rq[j] : acc_unkey<R>(ldd<COH>(&s.reqkey[c.sn[j]]));
                rq[j] = AC::add(rq[j], -(c.vals ? c.dn[j] : ldg(&s.dnet[c.sn[j]])));
            }
        }
#pragma unroll
        for (int j = 0; j < kBwPerLane; ++j) {
            if (c.p[j] < 0) continue;
            const A cand = AC::add(rq[j], -tp[j]);
            if (AC::lt(cand, m)) m = cand;
        }
    }
    // min is exact: any order gives the same value
    // (every lane shuffles; a small net's lanes take only partners in its group)
    const int gl = piece ? 32 : c.gl;
    for (int o = piece ? 16 : kBwLanes / 2; o > 0; o >>= 1) {
        const A other = shfl_x(m, o);
        if (o < gl && AC::lt(other, m)) m = other;
    }
    if (c.a >= 0 && (lane & (gl - 1)) == 0) {
        if (c.split) atomicMin(&s.reqkey[c.e], acc_key(m));
        else s.reqkey[c.e] = acc_key(m);
    }
}

// Required time of every pin that is not an endpoint, for sta_get_timing:
// a driver pin takes its net's required time, a combinational input its
// cell's output required time minus the cell delay (the addition of
// bwd_net).
template <typename R>
__global__ void k_pin_req(Topo t, State<R> s) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= t.n_pins) return;
    const int kind = ldg(&t.pin_kind[p]);
    if (kind == PK_ENDPOINT) return;
    if (kind == PK_COMB_IN) {
        const int sn = ldg(&t.sink_onet[p]);
        s.req[p] = Acc<R>::add(acc_unkey<R>(s.reqkey[sn]), -ldg(&s.dnet[sn]));
    } else {
        s.req[p] = acc_unkey<R>(s.reqkey[ldg(&t.pin_net[p])]);
    }
}

// Arrival of every combinational input pin: its driver's arrival plus its
// Elmore delay (the addition of fwd_cell), for sta_get_timing.
template <typename R>
__global__ void k_in_arr(Topo t, State<R> s) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= t.n_in) return;
    const int p = ldg(&t.lv_in_pin[j]);
    s.arr[p] = Acc<R>::add(s.arr[ldg(&t.lv_in_drv[j])], ldg(&s.tnet[p]));
}

// Slack = required time - arrival of every pin that is not an endpoint
// (Eq. (2)), for sta_get_timing; endpoints' slacks are k_ep_wns's.
template <typename R>
__global__ void k_pin_slack(Topo t, State<R> s) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= t.n_pins || ldg(&t.pin_kind[p]) == PK_ENDPOINT) return;
    s.slack[p] = Acc<R>::diff(s.req[p], s.arr[p]);
}

// Net weights from pin slacks, with momentum: the net-weighting scheme the
// paper compares against (Section II-C; the "w/o Path Extraction" ablation
// of Section IV).  The paper gives no formula; the reading: a net's
// criticality follows the worst slack over its pins, which is its driver
// pin's slack (a sink's slack is its required time minus the driver's
// arrival minus its Elmore delay, and the driver's required time is the
// least over its sinks of required time minus Elmore delay), formed here as
// k_pin_req and k_pin_slack form it; c = min(1, max(0, -slack) / |WNS|), 0
// when WNS = 0, and w <- alpha w + (1 - alpha)(1 + gamma c).  A thread per
// net; the nets of negative slack are counted with one integer atomic per
// block.
template <typename R>
__global__ void k_net_weights(Topo t, State<R> s, R alpha, R gamma) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    int crit = 0;
    if (e < t.n_nets) {
        const double wns = s.wns_tns[0];
        const R sl = Acc<R>::diff(acc_unkey<R>(s.reqkey[e]), s.arr[ldg(&t.net_ptr[e])]);
        R c = R(0);
        if (sl < R(0)) {
            crit = 1;
            if (wns < 0.0) c = min(R(1), -sl / (R)(-wns));
        }
        s.net_w[e] = alpha * s.net_w[e] + (R(1) - alpha) * (R(1) + gamma * c);
    }
    crit = __syncthreads_count(crit);
    if (threadIdx.x == 0 && crit > 0) atomicAdd(s.n_crit, crit);
}

template <typename R>
__global__ void k_fill(R *p, int n, R v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

// One launch per level (captured in a CUDA graph): a warp per task.
template <typename R>
__global__ void __launch_bounds__(kLvThreads) k_bwd_level(Topo t, State<R> s, int first, int n_small,
                                                          int n_piece) {
    pdl_trigger();
    const int w = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (w >= n_small + n_piece) return;
    SinkPre<R> c;
    sink_topo(t, first + w, threadIdx.x & 31, c);
    pdl_wait();  // everything below reads values earlier kernels wrote
    bwd_net<R, false>(s, c, threadIdx.x & 31, w >= n_small);
}


// ---------------------------------------------------------- WNS / TNS ---

constexpr int kRedThreads = 256;
constexpr int kRedFinal = 4 * kRedThreads;  // chunk partials the last block combines a round
constexpr int kCoopMaxBlocks = 1024;  // cap on the grid of a cooperative launch

// Endpoints (FF D and PO pins): arrival = the driver's arrival + the pin's
// Elmore delay, required time = T, slack = T - arrival, and whether the
// endpoint fails (slack < 0, the flags the extraction compacts into its list
// of failing endpoints); then WNS = min over endpoints with negative slack,
// TNS = their sum (FP64; Eqs. (2)-(4)).
// FP64 arithmetic is slow on this GPU, so the sums run as trees of fixed
// shape: a warp takes a chunk of kRedChunk endpoints (two per lane, then a
// butterfly over the lanes), and the last block to finish combines the
// chunk partials in rounds of kRedFinal, in chunk order: in a round, thread
// t adds chunks 4t .. 4t + 3 as pairs of pairs, a warp its lanes' sums by a
// butterfly, and one thread the 8 warps' sums as a pairwise tree.  The
// result does not depend on the grid or scheduling.  Needs the forward sweep only.
template <typename R>
__global__ void __launch_bounds__(kRedThreads) k_ep_wns(Topo t, State<R> s) {
    using AC = Acc<R>;
    using A = typename AC::T;
    static_assert(kRedChunk == 64, "two endpoints per lane");
    static_assert(kRedThreads == 256, "8 warp sums in the last block's tree");
    __shared__ bool last;
    __shared__ double2 wsum[kRedThreads / 32];
    chain_enter();
    const int lane = threadIdx.x & 31;
    const int n_chunks = div_up_dev(t.n_ep, kRedChunk);
    const int ch = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const A rq = acc_from_double<R>(*s.T);
    if (ch < n_chunks) {
        double mn[2] = {0.0, 0.0}, sm[2] = {0.0, 0.0};
        int2 pd[2];
        A ad[2];
        R tp[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int i = ch * kRedChunk + 32 * u + lane;
            if (i < t.n_ep) pd[u] = ldg(&t.ep_pd[i]);
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int i = ch * kRedChunk + 32 * u + lane;
            if (i < t.n_ep) {
                ad[u] = s.arr[pd[u].y];
                tp[u] = ldg(&s.tnet[pd[u].x]);
            }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int i = ch * kRedChunk + 32 * u + lane;
            if (i >= t.n_ep) continue;
            const A ap = AC::add(ad[u], tp[u]);
            const R sl = AC::diff(rq, ap);
            s.arr[pd[u].x] = ap;
            s.req[pd[u].x] = rq;
            s.slack[pd[u].x] = sl;
            const double v = (double)sl;
            s.ep_flag[i] = v < 0.0 ? 1 : 0;
            if (v < 0.0) {
                mn[u] = v;
                sm[u] = v;
            }
        }
        double m = fmin(mn[0], mn[1]), a = sm[0] + sm[1];
        for (int o = 16; o > 0; o >>= 1) {  // butterfly: the same pairs in every lane
            m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
            a += __shfl_xor_sync(0xffffffffu, a, o);
        }
        if (lane == 0) {
            s.red_part[2 * ch] = m;
            s.red_part[2 * ch + 1] = a;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(s.red_count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double bm = 0.0, bs = 0.0;
    const double2 *parts = reinterpret_cast<const double2 *>(s.red_part);
    for (int k0 = 0; k0 < n_chunks; k0 += kRedFinal) {
        double2 q[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int k = k0 + 4 * threadIdx.x + j;
            q[j] = k < n_chunks ? __ldcg(parts + k) : make_double2(0.0, 0.0);
        }
        double m = fmin(fmin(q[0].x, q[1].x), fmin(q[2].x, q[3].x));
        double a = (q[0].y + q[1].y) + (q[2].y + q[3].y);
        for (int o = 16; o > 0; o >>= 1) {
            m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
            a += __shfl_xor_sync(0xffffffffu, a, o);
        }
        if (lane == 0) wsum[threadIdx.x >> 5] = make_double2(m, a);
        __syncthreads();
        if (threadIdx.x == 0) {
            double2 w[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) w[k] = wsum[k];
#pragma unroll
            for (int h = 1; h < 8; h <<= 1)
#pragma unroll
                for (int k = 0; k < 8; k += 2 * h) w[k] = make_double2(fmin(w[k].x, w[k + h].x), w[k].y + w[k + h].y);
            bm = fmin(bm, w[0].x);
            bs += w[0].y;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        s.wns_tns[0] = bm;
        s.wns_tns[1] = bs;
        *s.red_count = 0u;
    }
}

// The whole backward sweep in one cooperative launch: levels
// from the deepest down to the startpoints' nets, a level's warp tasks on
// block j mod gridDim, a grid-wide barrier after each level.  A warp carries
// its first task of the next two levels: between its arrival at the barrier
// that closes level l and the wait, it loads the final values of its level
// l - 1 task and the topology of its level l - 2 task.
template <typename R>
__global__ void __launch_bounds__(kBwdThreads, 1) k_bwd_sweep(Topo t, State<R> s, GridSync gs) {
    const int lane = threadIdx.x & 31;
    const int w0 = blockIdx.x + (threadIdx.x >> 5) * gridDim.x;  // task j on block j mod gridDim
    const int wstride = (blockDim.x >> 5) * gridDim.x;
    auto task_of = [&](int l) {  // task w0 of level l, or -1
        if (l < 0) return -1;
        const int4 q = ldg(&t.bw_lv[l]);
        return w0 < q.y + q.z ? q.x + w0 : -1;
    };
    SinkPre<R> cur, nxt;
    sink_topo(t, task_of(t.depth), lane, cur);
    sink_vals(s, cur);
    sink_topo(t, task_of(t.depth - 1), lane, nxt);
    unsigned n = 0;
    for (int l = t.depth; l >= 0; --l) {
        const int4 q = ldg(&t.bw_lv[l]);  // (first task, small-net tasks, piece tasks)
        const int nt = q.y + q.z;
        if (w0 < nt) {
            bwd_net<R, true>(s, cur, lane, w0 >= q.y);
            for (int w = w0 + wstride; w < nt; w += wstride) {
                SinkPre<R> c;
                sink_topo(t, q.x + w, lane, c);
                bwd_net<R, true>(s, c, lane, w >= q.y);
            }
        }
        grid_arrive(gs);
        if (l > 0) {
            cur = nxt;
            sink_vals(s, cur);  // required times of levels above l are final
            sink_topo(t, task_of(l - 2), lane, nxt);
        }
        if (!grid_wait(gs, (++n) * gridDim.x)) return;
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
    if (bwd) ok = cudaMemsetAsync(s.reqkey, 0xff, sizeof(unsigned long long) * t.n_nets, cs) == cudaSuccess;
    for (int l = t.depth; bwd && l >= 0 && ok; --l) {
        const int ns = g->lv.bw_s_n[l], nb = g->lv.bw_b_n[l];
        if (ns + nb > 0) {
            launch_pdl(k_bwd_level<R>, div_up((int64_t)(ns + nb) * 32, kLvThreads), kLvThreads, cs, t, s,
                       g->lv.bw_s_lo[l], ns, nb);
            ++nk;
        }
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

// Blocks of a cooperative launch of `kernel` (smem bytes of dynamic shared
// memory a block) that are resident at once (at most kCoopMaxBlocks), cached
// per kernel; 0 if none.
template <typename K>
static int coop_grid(tdp_graph *g, K kernel, int threads, size_t smem = 0) {
    const void *key = reinterpret_cast<const void *>(kernel);
    for (auto &pr : g->coop_grid)
        if (pr.first == key) return pr.second;
    int nb = 0;
    if ((smem > 0 && cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                         cudaSuccess) ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        nb = 0;
    }
    const int grid = std::min(nb * g->n_sm, kCoopMaxBlocks);
    g->coop_grid.emplace_back(key, grid);
    return grid;
}

// gsync words: [0] forward sweep's barrier count, [1] sticky timeout status
// of both, [2] backward sweep's barrier count (the two sweeps may overlap
// when an extraction reruns the forward sweep)
template <typename R>
static tdp_status launch_sweep(tdp_graph *g, void (*kernel)(Topo, State<R>, GridSync), int grid,
                               int threads, KernelId id, cudaStream_t st, int count_word,
                               bool reset_count = true) {
    State<R> &s = state<R>(g);
    GridSync gs;
    gs.count = s.gsync + count_word;
    gs.status = s.gsync + 1;
    gs.timeout_ns = kSyncTimeoutNs;
    LaunchScope ls(g, id, 1, st);
    if (reset_count) TDP_CUDA(cudaMemsetAsync(gs.count, 0, sizeof(unsigned), st));
    TDP_CUDA(launch_coop(kernel, grid, threads, 0, st, g->topo, s, gs));
    return TDP_OK;
}

template <typename R>
static void (*fwd_kernel(int L))(Topo, State<R>, GridSync, const int *) {
    switch (L) {
        case 0: return k_fwd_sweep<R, 0>;
        case 3: return k_fwd_sweep<R, 3>;
        case 7: return k_fwd_sweep<R, 7>;
        case 15: return k_fwd_sweep<R, 15>;
        default: return k_fwd_sweep<R, 31>;
    }
}

// The single-launch forward sweep from level *from_dev (NULL: level 1);
// count_zeroed: the barrier word was set to 0 by the kernel before it (net
// RC), so the stream needs no memset.
template <typename R>
static tdp_status launch_fwd_sweep(tdp_graph *g, int grid, const int *from_dev, bool count_zeroed = false) {
    State<R> &s = state<R>(g);
    GridSync gs;
    gs.count = s.gsync;
    gs.status = s.gsync + 1;
    gs.timeout_ns = kSyncTimeoutNs;
    LaunchScope ls(g, KID_FWD_SWEEP, 1, g->stream);
    if (!count_zeroed) TDP_CUDA(cudaMemsetAsync(gs.count, 0, sizeof(unsigned), g->stream));
    TDP_CUDA(launch_coop(fwd_kernel<R>(g->list_L), grid, kFwdThreads, warp_list_smem<R>(g->list_L, kFwdThreads),
                         g->stream, g->topo, s, gs, from_dev));
    return TDP_OK;
}

// Forward sweep, building sidetrack lists of length g->list_L (0: none): one
// cooperative launch, or one graph replay of the level launches.  Run again,
// it writes the same arrival times.  after_rc: net RC was the stream's last
// kernel (it zeroes the sweep's barrier word).
template <typename R>
tdp_status forward_lists(tdp_graph *g, int leave_sms, bool after_rc) {
    State<R> &s = state<R>(g);
    if (g->list_L > 0 && !s.blist) TDP_TRY(dalloc(g, &s.blist, (size_t)g->topo.n_nets * kMaxK));
    if (g->single_launch) {
        if (g->topo.depth == 0) return TDP_OK;
        const int grid =
            coop_grid(g, fwd_kernel<R>(g->list_L), kFwdThreads, warp_list_smem<R>(g->list_L, kFwdThreads));
        if (grid > 0) return launch_fwd_sweep<R>(g, std::max(1, grid - leave_sms), nullptr, after_rc);
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

// reqkey := +inf keys (all ones) for the backward sweep, and its barrier
// count := 0: a kernel rather than memsets, so that the side stream holds
// only kernels
__global__ void k_bwd_reset(unsigned long long *reqkey, int n, unsigned *count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) reqkey[i] = ~0ull;
    if (i == 0) *count = 0u;
}

// Backward sweep: one cooperative launch, or one graph replay.  Nothing
// later in a timing iteration reads what it writes, so with the overlap on
// it runs on the graph's second stream from ev_bwd_go: in a full
// propagation, from the end of net RC on `sms` blocks (one an SM) beside the
// forward sweep on the other SMs, and on beside the endpoints, extraction,
// the pair update and the loss; else from the end of the forward sweep on
// bwd_share / 16 of its resident grid.  Serialised, on the graph's stream
// after the endpoints.  sta_join and every call that needs its results wait
// for it.
template <typename R>
static tdp_status backward(tdp_graph *g, int sms = 0) {
    cudaStream_t st = g->stream;
    if (g->overlap_bwd) {
        TDP_CUDA(cudaStreamWaitEvent(g->side, g->ev_bwd_go, 0));
        st = g->side;
    }
    bool done = false;
    if (g->single_launch) {
        // beside the forward sweep (sms, from bwd_split) or beside
        // extraction, the pair update and the loss (bwd_share / 16 of the
        // resident grid, 9/16 by default: 83 of 148 blocks; measured at 1.2M
        // cells, a step took 1.189, 1.157, 1.111, 1.135, 1.171 and 1.270 ms
        // for 7/16 to 12/16), the sweep leaves SMs to the rest
        int grid = coop_grid(g, k_bwd_sweep<R>, kBwdThreads);
        if (grid > 0 && g->overlap_bwd) grid = sms > 0 ? std::min(grid, sms) : std::max(1, grid * g->bwd_share / 16);
        if (grid > 0) {
            State<R> &s = state<R>(g);
            ++g->n_launch;
            k_bwd_reset<<<div_up(std::max(g->topo.n_nets, 1), 256), 256, 0, st>>>(s.reqkey, g->topo.n_nets,
                                                                                 s.gsync + 2);
            TDP_TRY(launch_sweep<R>(g, k_bwd_sweep<R>, grid, kBwdThreads, KID_BWD_SWEEP, st, 2, false));
            done = true;
        } else {
            g->single_launch = false;
        }
    }
    if (!done) {
        if (!g->bwd_graph) TDP_TRY(capture<R>(g, &g->bwd_graph, &g->bwd_graph_kernels, false, true, 0));
        LaunchScope ls(g, KID_BWD_SWEEP, g->bwd_graph_kernels, st);
        TDP_CUDA(cudaGraphLaunch(g->bwd_graph, st));
    }
    if (g->overlap_bwd) {
        TDP_CUDA(cudaEventRecord(g->ev_bwd, g->side));
        g->bwd_pending = true;
    }
    return TDP_OK;
}

// After the forward sweep: the endpoints and WNS / TNS, and the backward
// sweep (which reads no arrival and starts at once on the second stream).
template <typename R>
static tdp_status finish_sweeps(tdp_graph *g, bool bwd = true) {
    if (g->overlap_bwd && bwd) TDP_CUDA(cudaEventRecord(g->ev_bwd_go, g->stream));
    {
        LaunchScope ls(g, KID_EP_WNS);
        const int chunks = div_up(std::max(g->topo.n_ep, 1), kRedChunk);
        TDP_CUDA(launch_pdl(k_ep_wns<R>, div_up(chunks, kRedThreads / 32), kRedThreads, g->stream, g->topo,
                            state<R>(g)));
    }
    return bwd ? backward<R>(g) : TDP_OK;
}

// SMs for a backward sweep that starts with the forward sweep: the fewest
// with which its warps (kBwdThreads / 32 a block, one block an SM) take the
// tasks of all levels in at most kBwdRounds rounds a level on average, so
// that it ends about when the forward sweep and the rest of the iteration
// do; at most as many as leave every forward block at most two more chunks
// of a level than on all SMs.  Measured with 28-warp blocks at 1.2M cells
// (K = 16; 26 SMs here, 1.58 rounds a level): a step took 0.803, 0.789,
// 0.791, 0.793, 0.796 ms with 24, 26, 28, 30, 32 SMs (0.931 ms once with the
// backward sweep after the forward sweep); at 3.3M cells (K = 32; 43 SMs
// here), 2.94, 2.82, 2.82, 2.84, 2.85 ms with 36, 41, 44, 48, 52 SMs.
constexpr double kBwdRounds = 1.6;
static int bwd_split(const tdp_graph *g) {
    const Levels &lv = g->lv;
    const int n = std::max(g->n_sm, 2);
    int maxc = 1;
    for (size_t l = 1; l < lv.lvl_ptr.size(); ++l) maxc = std::max(maxc, div_up(lv.lvl_ptr[l] - lv.lvl_ptr[l - 1], 32));
    const int base = div_up(maxc, n);
    const int cap = std::max(1, std::min(n / 2, n - div_up(maxc, base + 2)));
    const int warps = kBwdThreads / 32;
    const double budget = kBwdRounds * (double)lv.bw_s_n.size();
    for (int x = 1; x < cap; ++x) {
        double rounds = 0.0;
        for (size_t l = 0; l < lv.bw_s_n.size(); ++l) rounds += div_up(lv.bw_s_n[l] + lv.bw_b_n[l], warps * x);
        if (rounds <= budget) return x;
    }
    return cap;
}

template tdp_status forward_lists<float>(tdp_graph *, int, bool);
template tdp_status forward_lists<double>(tdp_graph *, int, bool);

template <typename R>
tdp_status propagate_impl(tdp_graph *g, const R *x, const R *y, double T) {
    Topo &t = g->topo;
    State<R> &s = state<R>(g);
    const int nsb = div_up(t.n_nets, kRcThreads);
    join_side(g);  // the last backward sweep reads what this propagation rewrites
    g->inc_valid = false;
    {
        LaunchScope ls(g, KID_NET_RC);
        k_net_rc<R><<<nsb + t.n_big, kRcThreads, 0, g->stream>>>(t, s, x, y, T, (R)g->r, (R)g->c,
                                                                 (R)g->d0, nsb, Inc{});
    }
    TDP_LAUNCH_CHECK();
    if (g->list_L > 0 && !s.blist) TDP_TRY(dalloc(g, &s.blist, (size_t)t.n_nets * kMaxK));
    if (g->single_launch && g->overlap_bwd && t.depth > 0 && g->bwd_sms >= 0) {
        // required times need no arrival: the backward sweep starts now, on
        // its own SMs, and the forward sweep takes the others
        if (g->bwd_sms == 0) g->bwd_sms = bwd_split(g);
        TDP_CUDA(cudaEventRecord(g->ev_bwd_go, g->stream));
        TDP_TRY(backward<R>(g, g->bwd_sms));
        TDP_TRY(forward_lists<R>(g, g->bwd_sms, true));
        TDP_TRY(finish_sweeps<R>(g, false));
    } else {
        TDP_TRY(forward_lists<R>(g, 0, true));
        TDP_TRY(finish_sweeps<R>(g));
    }
    if (s.yprev) {  // incremental propagation is in use: keep these positions
        TDP_CUDA(cudaMemcpyAsync(s.xprev, x, sizeof(R) * t.n_cells, cudaMemcpyDeviceToDevice, g->stream));
        TDP_CUDA(cudaMemcpyAsync(s.yprev, y, sizeof(R) * t.n_cells, cudaMemcpyDeviceToDevice, g->stream));
        g->inc_valid = true;
    }
    g->inc_full = true;
    return TDP_OK;
}

template tdp_status propagate_impl<float>(tdp_graph *, const float *, const float *, double);
template tdp_status propagate_impl<double>(tdp_graph *, const double *, const double *, double);

// Buffers of incremental propagation, on its first use: the previous
// positions, the per-net stamps (zero: no call yet) and spans.
template <typename R>
static tdp_status inc_alloc(tdp_graph *g) {
    const Topo &t = g->topo;
    State<R> &s = state<R>(g);
    Inc &inc = g->inc;
    const size_t nn = (size_t)std::max(t.n_nets, 1);
    // each buffer once (a call that failed part way keeps what it got);
    // yprev last: its presence means the whole set is allocated
    if (!inc.stamp) TDP_TRY(dalloc(g, &inc.stamp, nn));
    if (!inc.span) TDP_TRY(dalloc(g, &inc.span, nn));
    if (!inc.lohi) TDP_TRY(dalloc(g, &inc.lohi, 3));
    if (!inc.cspan) TDP_TRY(dalloc(g, &inc.cspan, (size_t)std::max(t.n_cells, 1)));
    if (!inc.lvchg) TDP_TRY(dalloc(g, &inc.lvchg, (size_t)t.depth + 2));
    if (!inc.cnt) TDP_TRY(dalloc(g, &inc.cnt, 3));
    if (!s.xprev) TDP_TRY(dalloc(g, &s.xprev, (size_t)std::max(t.n_cells, 1)));
    TDP_TRY(dalloc(g, &s.yprev, (size_t)std::max(t.n_cells, 1)));
    TDP_CUDA(cudaMemsetAsync(inc.stamp, 0, sizeof(int32_t) * nn, g->stream));
    TDP_CUDA(cudaMemsetAsync(inc.cnt, 0, sizeof(unsigned long long) * 3, g->stream));
    inc.cur = 0;
    ++g->n_launch;
    k_inc_span<<<div_up((int)nn, 256), 256, 0, g->stream>>>(t, inc.span);
    TDP_LAUNCH_CHECK();
    ++g->n_launch;
    k_inc_cspan<<<div_up(std::max(t.n_cells, 1), 256), 256, 0, g->stream>>>(t, inc.span, inc.cspan);
    TDP_LAUNCH_CHECK();
    return TDP_OK;
}

// Incremental propagation: re-times only the nets of moved cells and the
// cells their changes reach (the same per-net and per-cell code as
// propagate_impl, so the same bits), then the endpoints and WNS / TNS and
// the backward sweep in full.  Re-times everything (and keeps the positions)
// when there is no valid previous propagation to start from.
template <typename R>
static tdp_status propagate_incremental_impl(tdp_graph *g, const R *x, const R *y, double T) {
    Topo &t = g->topo;
    State<R> &s = state<R>(g);
    if (!s.yprev) TDP_TRY(inc_alloc<R>(g));
    void (*kernel)(Topo, State<R>, GridSync, Inc);
    switch (g->list_L) {
        case 0: kernel = k_fwd_sweep_inc<R, 0>; break;
        case 3: kernel = k_fwd_sweep_inc<R, 3>; break;
        case 7: kernel = k_fwd_sweep_inc<R, 7>; break;
        case 15: kernel = k_fwd_sweep_inc<R, 15>; break;
        default: kernel = k_fwd_sweep_inc<R, 31>; break;
    }
    const int grid = g->single_launch ? coop_grid(g, kernel, kFwdThreads) : 0;
    const int grid_full = g->single_launch ? coop_grid(g, fwd_kernel<R>(g->list_L), kFwdThreads,
                                                       warp_list_smem<R>(g->list_L, kFwdThreads))
                                           : 0;
    if (!g->inc_valid || !g->propagated || grid == 0 || grid_full == 0 || g->lists_valid_L != g->list_L ||
        t.depth == 0)
        return propagate_impl<R>(g, x, y, T);
    join_side(g);  // the last backward sweep reads what this propagation rewrites
    g->inc_valid = false;
    Inc &inc = g->inc;
    if (inc.cur == INT_MAX) {  // stamps of earlier calls would alias: start over
        TDP_CUDA(cudaMemsetAsync(inc.stamp, 0, sizeof(int32_t) * std::max(t.n_nets, 1), g->stream));
        inc.cur = 0;
    }
    ++inc.cur;
    TDP_CUDA(cudaMemsetAsync(inc.lvchg, 0, sizeof(int32_t) * (t.depth + 2), g->stream));
    ++g->n_launch;
    k_inc_reset<<<1, 32, 0, g->stream>>>(inc);
    TDP_LAUNCH_CHECK();
    {
        LaunchScope ls(g, KID_INC_MOVED);
        k_inc_moved<R><<<div_up(std::max(t.n_cells, 1), 256), 256, 0, g->stream>>>(t, x, y, s.xprev, s.yprev,
                                                                                  inc);
    }
    TDP_LAUNCH_CHECK();
    const int nsb = div_up(t.n_nets, kRcThreads);
    {
        LaunchScope ls(g, KID_NET_RC);
        k_net_rc<R><<<nsb + t.n_big, kRcThreads, 0, g->stream>>>(t, s, x, y, T, (R)g->r, (R)g->c,
                                                                 (R)g->d0, nsb, inc);
    }
    TDP_LAUNCH_CHECK();
    {
        GridSync gs;
        gs.count = s.gsync;
        gs.status = s.gsync + 1;
        gs.timeout_ns = kSyncTimeoutNs;
        LaunchScope ls(g, KID_FWD_INC, 1, g->stream);
        TDP_CUDA(cudaMemsetAsync(gs.count, 0, sizeof(unsigned), g->stream));
        TDP_CUDA(launch_coop(kernel, grid, kFwdThreads, 0, g->stream, t, s, gs, inc));
    }
    // the levels after saturation, if the changes saturated (else it returns at once)
    TDP_TRY(launch_fwd_sweep<R>(g, grid_full, inc.lohi + 2));
    TDP_TRY(finish_sweeps<R>(g));
    g->inc_valid = true;
    g->inc_full = false;
    return TDP_OK;
}

template <typename R>
__global__ void k_acc_to_real(const typename Acc<R>::T *a, R *out, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = Acc<R>::val(a[i]);
}

template <typename R>
static tdp_status get_timing_impl(tdp_graph *g, R *arr, R *req, R *slack) {
    State<R> &s = state<R>(g);
    int n = g->topo.n_pins;
    join_side(g);
    g->n_launch += (arr || slack ? 1 : 0) + (req || slack ? 1 : 0) + (arr ? 1 : 0) + (req ? 1 : 0) + (slack ? 1 : 0);
    if ((arr || slack) && g->topo.n_in > 0)
        k_in_arr<R><<<div_up(g->topo.n_in, 256), 256, 0, g->stream>>>(g->topo, s);
    if (req || slack) k_pin_req<R><<<div_up(std::max(n, 1), 256), 256, 0, g->stream>>>(g->topo, s);
    if (arr) k_acc_to_real<R><<<div_up(n, 256), 256, 0, g->stream>>>(s.arr, arr, n);
    if (req) k_acc_to_real<R><<<div_up(n, 256), 256, 0, g->stream>>>(s.req, req, n);
    if (slack) k_pin_slack<R><<<div_up(std::max(n, 1), 256), 256, 0, g->stream>>>(g->topo, s);
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

static tdp_status propagate_common(tdp_graph *g, const void *x_dev, const void *y_dev, double clock_period_ps,
                                   double *wns_out, double *tns_out, bool incremental) {
    if (!g || !x_dev || !y_dev || !std::isfinite(clock_period_ps)) {
        set_error("%s: NULL graph or positions, or non-finite clock period",
                  incremental ? "sta_propagate_incremental" : "sta_propagate");
        return TDP_ERR_INVALID;
    }
    tdp_status st;
    if (g->prec == TDP_FP32) {
        const float *x = (const float *)x_dev, *y = (const float *)y_dev;
        st = incremental ? propagate_incremental_impl<float>(g, x, y, clock_period_ps)
                         : propagate_impl<float>(g, x, y, clock_period_ps);
    } else {
        const double *x = (const double *)x_dev, *y = (const double *)y_dev;
        st = incremental ? propagate_incremental_impl<double>(g, x, y, clock_period_ps)
                         : propagate_impl<double>(g, x, y, clock_period_ps);
    }
    if (st != TDP_OK) {  // a propagation that failed part way leaves no valid timing
        g->propagated = false;
        g->extracted = false;
        g->inc_valid = false;
        return st;
    }
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

extern "C" tdp_status sta_propagate(tdp_graph *g, const void *x_dev, const void *y_dev,
                                    double clock_period_ps, double *wns_out, double *tns_out) {
    return propagate_common(g, x_dev, y_dev, clock_period_ps, wns_out, tns_out, false);
}

extern "C" tdp_status sta_propagate_incremental(tdp_graph *g, const void *x_dev, const void *y_dev,
                                                double clock_period_ps, double *wns_out, double *tns_out) {
    return propagate_common(g, x_dev, y_dev, clock_period_ps, wns_out, tns_out, true);
}

extern "C" tdp_status sta_incremental_stats(tdp_graph *g, int64_t *stats_out) {
    if (!g || !stats_out) {
        set_error("sta_incremental_stats: NULL argument");
        return TDP_ERR_INVALID;
    }
    if (!g->propagated) {
        set_error("sta_incremental_stats: call sta_propagate_incremental first");
        return TDP_ERR_STATE;
    }
    const Topo &t = g->topo;
    if (g->inc_full || !g->inc.cnt) {
        const int64_t all[7] = {1, t.n_cells, t.n_comb, t.n_comb, t.depth > 0 ? 1 : 0, t.depth, 0};
        for (int i = 0; i < 7; ++i) stats_out[i] = all[i];
        return TDP_OK;
    }
    unsigned long long c[3];
    int32_t lh[3];
    TDP_CUDA(cudaMemcpyAsync(c, g->inc.cnt, sizeof(c), cudaMemcpyDeviceToHost, g->stream));
    TDP_CUDA(cudaMemcpyAsync(lh, g->inc.lohi, sizeof(lh), cudaMemcpyDeviceToHost, g->stream));
    TDP_CUDA(cudaStreamSynchronize(g->stream));
    stats_out[0] = 0;
    for (int i = 0; i < 3; ++i) stats_out[1 + i] = (int64_t)c[i];
    const bool none = lh[0] > lh[1];
    const bool sat = lh[2] <= t.depth;
    stats_out[4] = none ? 0 : lh[0];
    stats_out[5] = none ? -1 : (sat ? t.depth : std::min(lh[1], t.depth));
    stats_out[6] = sat ? lh[2] : 0;
    return TDP_OK;
}

extern "C" tdp_status sta_join(tdp_graph *g) {
    if (!g) {
        set_error("sta_join: NULL graph");
        return TDP_ERR_INVALID;
    }
    join_side(g);
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

namespace tdp {

// the net weights, allocated and set to 1 on first use (each buffer once:
// a call that failed part way keeps what it got)
template <typename R>
static tdp_status net_weights_ready(tdp_graph *g) {
    State<R> &s = state<R>(g);
    const int n = std::max(g->topo.n_nets, 1);
    if (!s.net_w) TDP_TRY(dalloc(g, &s.net_w, (size_t)n));
    if (!s.n_crit) TDP_TRY(dalloc(g, &s.n_crit, 1));
    if (!g->net_w_init) {
        ++g->n_launch;
        k_fill<R><<<div_up(n, 256), 256, 0, g->stream>>>(s.net_w, n, R(1));
        TDP_LAUNCH_CHECK();
        g->net_w_init = true;
    }
    return TDP_OK;
}

template <typename R>
static tdp_status net_weights_impl(tdp_graph *g, double alpha, double gamma, int64_t *n_crit_out) {
    State<R> &s = state<R>(g);
    const Topo &t = g->topo;
    TDP_TRY(net_weights_ready<R>(g));
    join_side(g);  // the nets' required times are the backward sweep's
    TDP_CUDA(cudaMemsetAsync(s.n_crit, 0, sizeof(int32_t), g->stream));
    if (t.n_nets > 0) {
        LaunchScope ls(g, KID_NET_WEIGHTS);
        k_net_weights<R><<<div_up(t.n_nets, 256), 256, 0, g->stream>>>(t, s, (R)alpha, (R)gamma);
    }
    TDP_LAUNCH_CHECK();
    if (n_crit_out) {
        int32_t h = 0;
        TDP_CUDA(cudaMemcpyAsync(&h, s.n_crit, sizeof(h), cudaMemcpyDeviceToHost, g->stream));
        TDP_TRY(check_sync_status(g));  // synchronises the stream
        *n_crit_out = h;
    }
    return TDP_OK;
}

}  // namespace tdp

extern "C" tdp_status net_weights_update(tdp_graph *g, double alpha, double gamma, int64_t *n_critical_out) {
    if (!g || !(alpha >= 0.0 && alpha <= 1.0) || !(gamma >= 0.0) || !std::isfinite(gamma)) {
        set_error("net_weights_update: NULL graph, alpha outside [0, 1] or gamma negative or not finite");
        return TDP_ERR_INVALID;
    }
    if (!g->propagated) {
        set_error("net_weights_update: call sta_propagate first");
        return TDP_ERR_STATE;
    }
    return g->prec == TDP_FP32 ? net_weights_impl<float>(g, alpha, gamma, n_critical_out)
                               : net_weights_impl<double>(g, alpha, gamma, n_critical_out);
}

extern "C" tdp_status net_weights_get(tdp_graph *g, void *w_dev) {
    if (!g || !w_dev) {
        set_error("net_weights_get: NULL graph or output");
        return TDP_ERR_INVALID;
    }
    const size_t n = (size_t)g->topo.n_nets;
    if (g->prec == TDP_FP32) {
        TDP_TRY(net_weights_ready<float>(g));
        TDP_CUDA(cudaMemcpyAsync(w_dev, g->s32.net_w, sizeof(float) * n, cudaMemcpyDeviceToDevice, g->stream));
    } else {
        TDP_TRY(net_weights_ready<double>(g));
        TDP_CUDA(cudaMemcpyAsync(w_dev, g->s64.net_w, sizeof(double) * n, cudaMemcpyDeviceToDevice, g->stream));
    }
    return TDP_OK;
}

extern "C" tdp_status net_weights_reset(tdp_graph *g) {
    if (!g) {
        set_error("net_weights_reset: NULL graph");
        return TDP_ERR_INVALID;
    }
    g->net_w_init = false;
    return g->prec == TDP_FP32 ? net_weights_ready<float>(g) : net_weights_ready<double>(g);
}

namespace tdp {
// every block waits for one more arrival than there are blocks
__global__ void k_wait_selftest(GridSync gs) { grid_sync(gs, gridDim.x + 1u); }
}  // namespace tdp

extern "C" tdp_status tdp_selftest_grid_wait(double timeout_ms, int32_t *gave_up_out) {
    if (!gave_up_out || !(timeout_ms > 0.0 && timeout_ms <= 1000.0)) {
        set_error("tdp_selftest_grid_wait: NULL output or timeout_ms outside (0, 1000]");
        return TDP_ERR_INVALID;
    }
    unsigned *w = nullptr;
    TDP_CUDA(cudaMalloc(&w, 2 * sizeof(unsigned)));
    GridSync gs;
    gs.count = w;
    gs.status = w + 1;
    gs.timeout_ns = (unsigned long long)(timeout_ms * 1e6);
    unsigned h[2] = {0u, 0u};
    cudaError_t e = cudaMemset(w, 0, 2 * sizeof(unsigned));
    if (e == cudaSuccess) e = launch_coop(k_wait_selftest, 2, 32, 0, (cudaStream_t)0, gs);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(h, w, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(w);
    if (e != cudaSuccess) {
        set_error("tdp_selftest_grid_wait: %s", cudaGetErrorString(e));
        return TDP_ERR_CUDA;
    }
    *gave_up_out = h[1] != 0u ? 1 : 0;
    return TDP_OK;
}
