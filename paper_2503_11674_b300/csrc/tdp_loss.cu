// Pin-to-pin attraction loss (Eq. (9); PP of Section III-D) and its adjoint.
//
//   PP = beta * sum over sinks s in P of w_s * ((x_s - x_d)^2 + (y_s - y_d)^2)
//
// or, as set by attraction_set_loss_kind, with the pair's HPWL or linear
// Euclidean distance in place of the quadratic term (the ablation of
// Section IV).
// with (x_d, y_d) the driver pin of s's net; pin coordinates are the cell
// position plus the pin offset.  Both passes take the sinks of P from the
// compacted, ascending list ppins, a thread per pair, so that no thread
// scans the other sinks of a net; the pairs of one net are consecutive
// there.  In the backward pass the first pair of a net of at most
// kBigFanout sinks sums its net's pin gradients for the driver, in FP64, in
// pin order; a larger net is a warp's (the static list of larger nets,
// skipped without a pair), which walks its sinks and sums in a fixed order.
//
//   k_pp_fwd       terms in the working precision, FP64 total; fixed grid and
//                  fixed-order block / grid reduction (deterministic)
//   k_pp_bwd_net   pin gradients 2 beta w (p_s - p_d) of the sinks in P,
//                  minus their sum on each net's driver, into the pins' slots
//                  in the cell -> pins order (slots outside P stay zero)
//   k_pp_bwd_cell  per cell of the compacted list pcells, the FP64 sum of its
//                  pins' slots times the incoming gradient scale (fixed cells
//                  0); every other cell's gradient is 0
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

// Pair term of sink pin p, with a the driver pin of its net.
template <typename R>
__device__ __forceinline__ R pin_pp(const Topo &t, const State<R> &s, const R *x, const R *y, int p, int a,
                                    int kind) {
    const int cd = t.pin_cell[a];
    const R xd = x[cd] + s.pin_dx[a], yd = y[cd] + s.pin_dy[a];
    const int cs = t.pin_cell[p];
    const R dx = x[cs] + s.pin_dx[p] - xd;
    const R dy = y[cs] + s.pin_dy[p] - yd;
    return s.w[p] * pair_term(dx, dy, kind);
}

template <typename R>
__global__ void __launch_bounds__(kLossThreads) k_pp_fwd(Topo t, State<R> s, const R *__restrict__ x,
                                                         const R *__restrict__ y, double beta,
                                                         int kind, double *loss) {
    __shared__ double sh[kLossThreads / 32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int np = s.pcnt[0];
    double acc = 0.0;
    for (int i = blockIdx.x * kLossThreads + threadIdx.x; i < np; i += gridDim.x * kLossThreads) {
        const int p = s.ppins[i];
        acc += (double)pin_pp(t, s, x, y, p, t.net_ptr[t.pin_net[p]], kind);
    }
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
    if (last && threadIdx.x < 32) {
        __threadfence();
        const volatile double *part = s.loss_part;
        double v = 0.0;
        for (int k = lane; k < (int)gridDim.x; k += 32) v += part[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) {
            *loss = beta * v;
            *s.loss_count = 0u;
        }
    }
}

// Pin gradients of one net.  Lanes [first, first+step) share the net when it
// is large; the driver's sum is returned to the caller (partial per lane).
template <typename R>
__device__ __forceinline__ void net_grad(const Topo &t, State<R> &s, const R *x, const R *y,
                                         int a, int b, int first, int step, double beta, int kind,
                                         double &sx, double &sy) {
    const int cd = t.pin_cell[a];
    const R xd = x[cd] + s.pin_dx[a], yd = y[cd] + s.pin_dy[a];
    for (int p = a + 1 + first; p < b; p += step) {
        if (!s.in_p[p]) continue;
        const int cs = t.pin_cell[p];
        const R k = (R)beta * s.w[p];
        R ux, uy;
        pair_grad(x[cs] + s.pin_dx[p] - xd, y[cs] + s.pin_dy[p] - yd, kind, ux, uy);
        const R gx = k * ux;
        const R gy = k * uy;
        sx += (double)gx;
        sy += (double)gy;
        const int slot = t.slot_of_pin[p];
        s.gslot[2 * slot] = gx;
        s.gslot[2 * slot + 1] = gy;
    }
}

// Gradient of the pair term of sink pin p (driver pin a) with respect to the
// sink's position, times beta w (the arithmetic of net_grad).
template <typename R>
__device__ __forceinline__ void pin_grad(const Topo &t, const State<R> &s, const R *x, const R *y, int p, int a,
                                         double beta, int kind, R &gx, R &gy) {
    const int cd = t.pin_cell[a];
    const R xd = x[cd] + s.pin_dx[a], yd = y[cd] + s.pin_dy[a];
    const int cs = t.pin_cell[p];
    const R k = (R)beta * s.w[p];
    R ux, uy;
    pair_grad(x[cs] + s.pin_dx[p] - xd, y[cs] + s.pin_dy[p] - yd, kind, ux, uy);
    gx = k * ux;
    gy = k * uy;
}

// warp tasks: warps [0, npw) take 32 consecutive pairs of ppins (a lane per
// pair; pairs of larger nets are left to their net's warp), warps
// [npw, npw + n_big) one larger net each
template <typename R>
__global__ void __launch_bounds__(256) k_pp_bwd_net(Topo t, State<R> s, const R *__restrict__ x,
                                                    const R *__restrict__ y, double beta, int kind) {
    const int lane = threadIdx.x & 31;
    const int np = s.pcnt[0];
    const int npw = (np + 31) >> 5;
    const int tasks = npw + t.n_big;
    const int nwarps = (int)((gridDim.x * (size_t)blockDim.x) >> 5);
    for (int task = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5); task < tasks; task += nwarps) {
        if (task < npw) {
            const int i = task * 32 + lane;
            if (i >= np) continue;
            const int p = s.ppins[i];
            const int e = t.pin_net[p];
            const int a = t.net_ptr[e];
            if (t.net_ptr[e + 1] - a - 1 > kBigFanout) continue;  // its net's warp
            R gx, gy;
            pin_grad(t, s, x, y, p, a, beta, kind, gx, gy);
            const int slot = t.slot_of_pin[p];
            s.gslot[2 * slot] = gx;
            s.gslot[2 * slot + 1] = gy;
            if (i > 0 && t.pin_net[s.ppins[i - 1]] == e) continue;
            // the net's first pair: the driver's gradient, minus the sum of
            // the net's pin gradients in pin order (at most kBigFanout)
            double sx = (double)gx, sy = (double)gy;
            for (int j = i + 1; j < np; ++j) {
                const int q = s.ppins[j];
                if (t.pin_net[q] != e) break;
                R qx, qy;
                pin_grad(t, s, x, y, q, a, beta, kind, qx, qy);
                sx += (double)qx;
                sy += (double)qy;
            }
            const int ds = t.slot_of_pin[a];
            s.gslot[2 * ds] = (R)(-sx);
            s.gslot[2 * ds + 1] = (R)(-sy);
        } else {
            const int e = t.big_nets[task - npw];
            if (!s.net_pf[e]) continue;  // warp-uniform
            const int a = t.net_ptr[e];
            double sx = 0.0, sy = 0.0;
            net_grad(t, s, x, y, a, t.net_ptr[e + 1], lane, 32, beta, kind, sx, sy);
            for (int o = 16; o > 0; o >>= 1) {
                sx += __shfl_xor_sync(0xffffffffu, sx, o);
                sy += __shfl_xor_sync(0xffffffffu, sy, o);
            }
            if (lane != 0) continue;
            const int ds = t.slot_of_pin[a];
            s.gslot[2 * ds] = (R)(-sx);
            s.gslot[2 * ds + 1] = (R)(-sy);
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(256) k_pp_bwd_cell(Topo t, State<R> s, const double *gscale,
                                                     R *__restrict__ gx, R *__restrict__ gy) {
    const int nc = s.pcnt[1];
    const double g = gscale ? *gscale : 1.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
        const int c = s.pcells[i];
        double ax = 0.0, ay = 0.0;
        if (!t.cell_fixed[c]) {
            for (int k = t.cp_ptr[c]; k < t.cp_ptr[c + 1]; ++k) {
                ax += (double)s.gslot[2 * k];
                ay += (double)s.gslot[2 * k + 1];
            }
            ax *= g;
            ay *= g;
        }
        gx[c] = (R)ax;
        gy[c] = (R)ay;
    }
}

template <typename R>
tdp_status loss_fwd_impl(tdp_graph *g, const R *x, const R *y, double beta, double *loss) {
    LaunchScope ls(g, KID_PP_FWD);
    k_pp_fwd<R><<<kLossBlocks, kLossThreads, 0, g->stream>>>(g->topo, state<R>(g), x, y, beta, g->loss_kind,
                                                              loss);
    TDP_LAUNCH_CHECK();
    return TDP_OK;
}

template <typename R>
tdp_status loss_bwd_impl(tdp_graph *g, const R *x, const R *y, double beta, const double *gs,
                         R *gx, R *gy) {
    Topo &t = g->topo;
    State<R> &s = state<R>(g);
    TDP_CUDA(cudaMemsetAsync(gx, 0, sizeof(R) * t.n_cells, g->stream));
    TDP_CUDA(cudaMemsetAsync(gy, 0, sizeof(R) * t.n_cells, g->stream));
    {
        LaunchScope ls(g, KID_PP_BWD_NET);
        k_pp_bwd_net<R><<<kLossBlocks, 256, 0, g->stream>>>(t, s, x, y, beta, g->loss_kind);
    }
    {
        LaunchScope ls(g, KID_PP_BWD_CELL);
        k_pp_bwd_cell<R><<<kLossBlocks, 256, 0, g->stream>>>(t, s, gs, gx, gy);
    }
    TDP_LAUNCH_CHECK();
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

extern "C" tdp_status attraction_set_loss_kind(tdp_graph *g, tdp_loss_kind kind) {
    if (!g || (kind != TDP_LOSS_QUADRATIC && kind != TDP_LOSS_HPWL && kind != TDP_LOSS_EUCLID)) {
        set_error("attraction_set_loss_kind: NULL graph or unknown kind");
        return TDP_ERR_INVALID;
    }
    g->loss_kind = (int)kind;
    return TDP_OK;
}
