// Pin-to-pin attraction loss (Eq. (9); PP of Section III-D) and its adjoint.
//
//   PP = beta * sum over sinks s in P of w_s * ((x_s - x_d)^2 + (y_s - y_d)^2)
//
// or, as set by attraction_set_loss_kind, with the pair's HPWL or linear
// Euclidean distance in place of the quadratic term (the ablation of
// Section IV), with (x_d, y_d) the driver pin of s's net; pin coordinates
// are the cell position plus the pin offset.  Both passes read the pair
// records (State::pr_*, rebuilt after each change of P, in the ascending
// order of the sinks of P, so that the pairs of one net are consecutive):
// a record, then the two cells' positions, a thread per pair.
//
//   k_pp_fwd       terms in the working precision, FP64 total; fixed grid and
//                  fixed-order block / grid reduction (deterministic)
//   k_pp_bwd_net   pin gradients beta w dQ/dp_s of the sinks in P into their
//                  slots in the cell -> pins order, and minus their sum, in
//                  FP64, on each net's driver: the first pair of a net of at
//                  most kBigFanout sinks sums its net's pairs in pin order; a
//                  larger net holding a pair is a warp's (lanes strided over
//                  its pairs, then a butterfly), in a fixed order either way.
//                  Slots outside P stay zero
//   (attraction_loss_fwd_bwd runs k_pp_bwd_net with the loss terms added,
//   the total formed as k_pp_fwd forms it, then k_pp_bwd_cell: two launches)
//   k_pp_bwd_cell  per cell of the compacted list pcells, the FP64 sum of its
//                  pins' slots times the incoming gradient scale (fixed cells
//                  0); in the same launch, 0 for every other cell
#include "tdp_internal.cuh"

namespace tdp {

constexpr int kLossBlocks = 148 * 4;
constexpr int kLossThreads = 256;

// Pair distance term (kind 0: Q(i,j) of Eq. (9); 1: |dx| + |dy|; 2:
// sqrt(dx^2 + dy^2), the ablation's alternatives) and its gradient with
// respect to the sink's position, per unit weight and beta.
template <typename R>
__device__ __forceinline__ R pair_term(R dx, R dy, int kind) {
    if (kind == 1) return fabs(dx) + fabs(dy);
    if (kind == 2) return sqrt(dx * dx + dy * dy);
    return dx * dx + dy * dy;
}
template <typename R>
__device__ __forceinline__ void pair_grad(R dx, R dy, int kind, R &gx, R &gy) {
    if (kind == 1) {
        gx = (R)((dx > R(0)) - (dx < R(0)));
        gy = (R)((dy > R(0)) - (dy < R(0)));
    } else if (kind == 2) {
        const R d = sqrt(dx * dx + dy * dy);
        gx = d > R(0) ? dx / d : R(0);
        gy = d > R(0) ? dy / d : R(0);
    } else {
        gx = R(2) * dx;
        gy = R(2) * dy;
    }
}

// a pin's gradient slot (x, y) as one vector access
__device__ __forceinline__ void put_slot(float *g, int slot, float a, float b) {
    reinterpret_cast<float2 *>(g)[slot] = make_float2(a, b);
}
__device__ __forceinline__ void put_slot(double *g, int slot, double a, double b) {
    reinterpret_cast<double2 *>(g)[slot] = make_double2(a, b);
}
__device__ __forceinline__ float2 get_slot(const float *g, int slot) { return reinterpret_cast<const float2 *>(g)[slot]; }
__device__ __forceinline__ double2 get_slot(const double *g, int slot) {
    return reinterpret_cast<const double2 *>(g)[slot];
}

// the four offsets of pair record i (sink x, y, driver x, y)
__device__ __forceinline__ void pair_offsets(const float *o, int i, float (&v)[4]) {
    const float4 q = __ldg(reinterpret_cast<const float4 *>(o) + i);
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = q.w;
}
__device__ __forceinline__ void pair_offsets(const double *o, int i, double (&v)[4]) {
    const double2 q0 = __ldg(reinterpret_cast<const double2 *>(o) + 2 * i);
    const double2 q1 = __ldg(reinterpret_cast<const double2 *>(o) + 2 * i + 1);
    v[0] = q0.x;
    v[1] = q0.y;
    v[2] = q1.x;
    v[3] = q1.y;
}

// The sink-minus-driver pin vector of pair record i (record r): the pin
// coordinates are the cell position plus the pin offset.
template <typename R>
__device__ __forceinline__ void pair_vec(const State<R> &s, const R *x, const R *y, int i, const int4 &r, R &dx,
                                         R &dy) {
    R o[4];
    pair_offsets(s.pr_o, i, o);
    const R xd = x[r.y] + o[2], yd = y[r.y] + o[3];
    dx = x[r.x] + o[0] - xd;
    dy = y[r.x] + o[1] - yd;
}

// The loss total from each thread's FP64 partial, in a fixed order: a
// butterfly in the warp, the warps of the block in order, then the last
// block to finish adds the blocks' partials (thread t the partials t,
// t + kLossThreads, ... in order, then a butterfly in the warp and the warps
// in order), so the result depends on neither scheduling nor timing.  The
// last block issues its loads of the partials before it adds any.
template <typename R>
__device__ __forceinline__ void loss_total(const State<R> &s, double acc, double beta, double *loss) {
    constexpr int kPer = (kLossBlocks + kLossThreads - 1) / kLossThreads;  // partials a thread
    __shared__ double sh[kLossThreads / 32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) sh[wib] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int k = 0; k < kLossThreads / 32; ++k) b += sh[k];
        s.loss_part[blockIdx.x] = b;
        __threadfence();
        last = atomicAdd(s.loss_count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double v = 0.0;
    for (int k0 = 0; k0 < (int)gridDim.x; k0 += kPer * kLossThreads) {
        double q[kPer];
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int k = k0 + j * kLossThreads + (int)threadIdx.x;
            q[j] = k < (int)gridDim.x ? __ldcg(&s.loss_part[k]) : 0.0;
        }
#pragma unroll
        for (int j = 0; j < kPer; ++j) v += q[j];
    }
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[wib] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int k = 0; k < kLossThreads / 32; ++k) b += sh[k];
        *loss = beta * b;
        *s.loss_count = 0u;
    }
}

template <typename R>
__global__ void __launch_bounds__(kLossThreads) k_pp_fwd(Topo t, State<R> s, const R *__restrict__ x,
                                                         const R *__restrict__ y, double beta,
                                                         int kind, double *loss) {
    chain_enter();
    const int np = s.pcnt[0];
    double acc = 0.0;
    for (int i = blockIdx.x * kLossThreads + threadIdx.x; i < np; i += gridDim.x * kLossThreads) {
        const int4 r = __ldg(&s.pr_a[i]);
        R dx, dy;
        pair_vec(s, x, y, i, r, dx, dy);
        acc += (double)(__ldg(&s.pr_w[i]) * pair_term(dx, dy, kind));
    }
    loss_total(s, acc, beta, loss);
}

// beta w dQ/dp_s of a pair from its pin vector (dx, dy) and weight
template <typename R>
__device__ __forceinline__ void vec_grad(R dx, R dy, R w, double beta, int kind, R &gx, R &gy) {
    R ux, uy;
    const R k = (R)beta * w;
    pair_grad(dx, dy, kind, ux, uy);
    gx = k * ux;
    gy = k * uy;
}

// Gradient of pair record i's term with respect to the sink's position,
// beta w dQ/dp_s.
template <typename R>
__device__ __forceinline__ void rec_grad(const State<R> &s, const R *x, const R *y, int i, const int4 &r,
                                         double beta, int kind, R &gx, R &gy) {
    R dx, dy;
    pair_vec(s, x, y, i, r, dx, dy);
    vec_grad(dx, dy, __ldg(&s.pr_w[i]), beta, kind, gx, gy);
}

// warp tasks: warps [0, npw) take 32 consecutive pair records (a lane per
// pair), warps [npw, npw + pr_nbig) one larger net each.  FWD (the fused
// forward + backward call): each lane also adds its record's term to the
// loss, and the grid forms the total as k_pp_fwd does.  Launched on the same
// grid (kLossBlocks x kLossThreads), a thread visits its records in the
// order k_pp_fwd's thread of the same index does, so the total has the
// same bits.
template <typename R, bool FWD>
__global__ void __launch_bounds__(kLossThreads) k_pp_bwd_net(Topo t, State<R> s, const R *__restrict__ x,
                                                             const R *__restrict__ y, double beta, int kind,
                                                             double *loss) {
    chain_enter();
    const int lane = threadIdx.x & 31;
    const int np = s.pcnt[0];
    const int npw = (np + 31) >> 5;
    const int tasks = npw + *s.pr_nbig;
    const int nwarps = (int)((gridDim.x * (size_t)blockDim.x) >> 5);
    double acc = 0.0;
    for (int task = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5); task < tasks; task += nwarps) {
        if (task < npw) {
            const int i = task * 32 + lane;
            if (i >= np) continue;
            const int4 r = __ldg(&s.pr_a[i]);
            R dx, dy, gx, gy;
            pair_vec(s, x, y, i, r, dx, dy);
            const R w = __ldg(&s.pr_w[i]);
            if constexpr (FWD) acc += (double)(w * pair_term(dx, dy, kind));
            vec_grad(dx, dy, w, beta, kind, gx, gy);
            put_slot(s.gslot, r.z, gx, gy);
            if (r.w < 0) continue;
            // the first pair of a net of at most kBigFanout sinks: the driver's
            // gradient, minus the sum of the net's pin gradients in pin order
            double sx = (double)gx, sy = (double)gy;
            const int n = __ldg(&s.pr_n[i]);
            for (int j = i + 1; j < i + n; ++j) {
                const int4 q = __ldg(&s.pr_a[j]);
                R qx, qy;
                rec_grad(s, x, y, j, q, beta, kind, qx, qy);
                sx += (double)qx;
                sy += (double)qy;
            }
            put_slot(s.gslot, r.w, (R)(-sx), (R)(-sy));
        } else {
            const int4 big = __ldg(&s.pr_big[task - npw]);  // (first record, pairs, driver slot)
            double sx = 0.0, sy = 0.0;
            for (int j = big.x + lane; j < big.x + big.y; j += 32) {
                const int4 q = __ldg(&s.pr_a[j]);
                R qx, qy;
                rec_grad(s, x, y, j, q, beta, kind, qx, qy);
                sx += (double)qx;
                sy += (double)qy;
            }
            for (int o = 16; o > 0; o >>= 1) {
                sx += __shfl_xor_sync(0xffffffffu, sx, o);
                sy += __shfl_xor_sync(0xffffffffu, sy, o);
            }
            if (lane != 0) continue;
            put_slot(s.gslot, big.z, (R)(-sx), (R)(-sy));
        }
    }
    if constexpr (FWD) loss_total(s, acc, beta, loss);
}

// Two roles in one launch, on disjoint cells: blocks [0, kCellBlocks) take
// the compacted list pcells (the cells with a pin in a pair) densely, so that
// the FP64 sums run on full warps; the other blocks write zero gradients to
// every cell without a pin in a pair, a cell a thread.
constexpr int kCellBlocks = 148 * 4;

template <typename R>
__global__ void __launch_bounds__(256) k_pp_bwd_cell(Topo t, State<R> s, const double *gscale,
                                                     R *__restrict__ gx, R *__restrict__ gy) {
    chain_enter();
    if (blockIdx.x < kCellBlocks) {
        const int nc = s.pcnt[1];
        const double g = gscale ? *gscale : 1.0;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += kCellBlocks * blockDim.x) {
            const int c = s.pcells[i];
            double ax = 0.0, ay = 0.0;
            if (!t.cell_fixed[c]) {
                for (int k = t.cp_ptr[c]; k < t.cp_ptr[c + 1]; ++k) {
                    const auto v = get_slot(s.gslot, k);
                    ax += (double)v.x;
                    ay += (double)v.y;
                }
                ax *= g;
                ay *= g;
            }
            gx[c] = (R)ax;
            gy[c] = (R)ay;
        }
        return;
    }
    // one cell a thread: a warp's stores cover 32 consecutive cells
    const int c = (blockIdx.x - kCellBlocks) * blockDim.x + threadIdx.x;
    if (c < t.n_cells && !s.cell_pf[c]) {
        gx[c] = R(0);
        gy[c] = R(0);
    }
}

template <typename R>
tdp_status loss_fwd_impl(tdp_graph *g, const R *x, const R *y, double beta, double *loss) {
    LaunchScope ls(g, KID_PP_FWD);
    TDP_CUDA(launch_pdl(k_pp_fwd<R>, kLossBlocks, kLossThreads, g->stream, g->topo, state<R>(g), x, y, beta,
                        g->loss_kind, loss));
    return TDP_OK;
}

template <typename R>
tdp_status loss_bwd_impl(tdp_graph *g, const R *x, const R *y, double beta, const double *gs,
                         R *gx, R *gy) {
    Topo &t = g->topo;
    State<R> &s = state<R>(g);
    {
        LaunchScope ls(g, KID_PP_BWD_NET);
        TDP_CUDA(launch_pdl(k_pp_bwd_net<R, false>, kLossBlocks, kLossThreads, g->stream, t, s, x, y, beta,
                            g->loss_kind, (double *)nullptr));
    }
    {
        LaunchScope ls(g, KID_PP_BWD_CELL);
        const int zero_blocks = div_up(std::max(t.n_cells, 1), 256);
        TDP_CUDA(launch_pdl(k_pp_bwd_cell<R>, kCellBlocks + zero_blocks, 256, g->stream, t, s, gs, gx, gy));
    }
    return TDP_OK;
}

// attraction_loss_fwd_bwd: the per-pair pass computes the loss terms with
// the pin gradients (k_pp_bwd_net<R, true>), then the cell pass
template <typename R>
static tdp_status loss_fwd_bwd_impl(tdp_graph *g, const R *x, const R *y, double beta, const double *gs,
                                    double *loss, R *gx, R *gy) {
    Topo &t = g->topo;
    State<R> &s = state<R>(g);
    {
        LaunchScope ls(g, KID_PP_FWD_BWD);
        TDP_CUDA(launch_pdl(k_pp_bwd_net<R, true>, kLossBlocks, kLossThreads, g->stream, t, s, x, y, beta,
                            g->loss_kind, loss));
    }
    {
        LaunchScope ls(g, KID_PP_BWD_CELL);
        const int zero_blocks = div_up(std::max(t.n_cells, 1), 256);
        TDP_CUDA(launch_pdl(k_pp_bwd_cell<R>, kCellBlocks + zero_blocks, 256, g->stream, t, s, gs, gx, gy));
    }
    return TDP_OK;
}

template tdp_status loss_fwd_impl<float>(tdp_graph *, const float *, const float *, double, double *);
template tdp_status loss_fwd_impl<double>(tdp_graph *, const double *, const double *, double, double *);
template tdp_status loss_bwd_impl<float>(tdp_graph *, const float *, const float *, double,
                                         const double *, float *, float *);
template tdp_status loss_bwd_impl<double>(tdp_graph *, const double *, const double *, double,
                                          const double *, double *, double *);

// ------------------------------------------------------------------ scan ---
constexpr int kScanThreads = 1024, kScanItems = 4, kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ long long block_excl_scan(long long v, long long *sh, long long &total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        long long s = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        sh[lane] = s;
    }
    __syncthreads();
    total = sh[(blockDim.x >> 5) - 1];
    long long before = w > 0 ? sh[w - 1] : 0;
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const int32_t *in, int64_t n, long long *tile_sum) {
    __shared__ long long sh[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    long long v = 0;
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) v += in[base + k];
    long long total;
    block_excl_scan(v, sh, total);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_sums(long long *tile_sum, int nt, int64_t *out_total) {
    __shared__ long long sh[32];
    long long carry = 0;
    for (int b = 0; b < nt; b += kScanThreads) {
        const int i = b + threadIdx.x;
        long long v = i < nt ? tile_sum[i] : 0;
        long long total;
        long long ex = block_excl_scan(v, sh, total);
        if (i < nt) tile_sum[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) *out_total = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const int32_t *in, int64_t n,
                                                             const long long *tile_off, int64_t *out) {
    __shared__ long long sh[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    int32_t v[kScanItems];
    long long sum = 0;
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < n ? in[base + k] : 0;
        sum += v[k];
    }
    long long total;
    long long run = block_excl_scan(sum, sh, total) + tile_off[blockIdx.x];
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
}

tdp_status scan_i32_to_i64(tdp_graph *g, const int32_t *in, int64_t *out, int64_t n, cudaStream_t st) {
    g->n_launch += 3;
    const int nt = div_up(std::max<int64_t>(n, 1), kScanTile);
    long long *tile = nullptr;
    if (dmalloc_async(&tile, sizeof(long long) * nt, st) != cudaSuccess) {
        set_error("scan: temporary allocation failed");
        return TDP_ERR_OOM;
    }
    k_scan_tiles<<<nt, kScanThreads, 0, st>>>(in, n, tile);
    k_scan_sums<<<1, kScanThreads, 0, st>>>(tile, nt, out + n);
    k_scan_apply<<<nt, kScanThreads, 0, st>>>(in, n, tile, out);
    cudaFreeAsync(tile, st);
    TDP_LAUNCH_CHECK();
    return TDP_OK;
}

}  // namespace tdp

using namespace tdp;

extern "C" tdp_status attraction_loss_fwd(tdp_graph *g, const void *x_dev, const void *y_dev,
                                          double beta, double *loss_dev) {
    if (!g || !x_dev || !y_dev || !loss_dev || !std::isfinite(beta)) {
        set_error("attraction_loss_fwd: NULL argument or non-finite beta");
        return TDP_ERR_INVALID;
    }
    return g->prec == TDP_FP32
               ? loss_fwd_impl<float>(g, (const float *)x_dev, (const float *)y_dev, beta, loss_dev)
               : loss_fwd_impl<double>(g, (const double *)x_dev, (const double *)y_dev, beta, loss_dev);
}

extern "C" tdp_status attraction_loss_bwd(tdp_graph *g, const void *x_dev, const void *y_dev,
                                          double beta, const double *grad_scale_dev, void *gx_dev,
                                          void *gy_dev) {
    if (!g || !x_dev || !y_dev || !gx_dev || !gy_dev || !std::isfinite(beta)) {
        set_error("attraction_loss_bwd: NULL argument or non-finite beta");
        return TDP_ERR_INVALID;
    }
    return g->prec == TDP_FP32
               ? loss_bwd_impl<float>(g, (const float *)x_dev, (const float *)y_dev, beta,
                                      grad_scale_dev, (float *)gx_dev, (float *)gy_dev)
               : loss_bwd_impl<double>(g, (const double *)x_dev, (const double *)y_dev, beta,
                                       grad_scale_dev, (double *)gx_dev, (double *)gy_dev);
}

extern "C" tdp_status attraction_loss_fwd_bwd(tdp_graph *g, const void *x_dev, const void *y_dev, double beta,
                                              const double *grad_scale_dev, double *loss_dev, void *gx_dev,
                                              void *gy_dev) {
    if (!g || !x_dev || !y_dev || !loss_dev || !gx_dev || !gy_dev || !std::isfinite(beta)) {
        set_error("attraction_loss_fwd_bwd: NULL argument or non-finite beta");
        return TDP_ERR_INVALID;
    }
    return g->prec == TDP_FP32
               ? loss_fwd_bwd_impl<float>(g, (const float *)x_dev, (const float *)y_dev, beta, grad_scale_dev,
                                          loss_dev, (float *)gx_dev, (float *)gy_dev)
               : loss_fwd_bwd_impl<double>(g, (const double *)x_dev, (const double *)y_dev, beta, grad_scale_dev,
                                           loss_dev, (double *)gx_dev, (double *)gy_dev);
}

extern "C" tdp_status attraction_set_loss_kind(tdp_graph *g, tdp_loss_kind kind) {
    if (!g || (kind != TDP_LOSS_QUADRATIC && kind != TDP_LOSS_HPWL && kind != TDP_LOSS_EUCLID)) {
        set_error("attraction_set_loss_kind: NULL graph or unknown kind");
        return TDP_ERR_INVALID;
    }
    g->loss_kind = (int)kind;
    return TDP_OK;
}
