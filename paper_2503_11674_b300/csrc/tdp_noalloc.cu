// attraction_loss_fwd_noalloc: the attraction loss forward pass for callers
// that cannot allocate device memory.
//
// Some callers may not call cudaMalloc (or any routine that allocates): code
// running inside a memory budget fixed in advance, code that hands all device
// memory to its own pool, or code that must not trigger allocation after
// start-up.  This entry point takes every input and the output as caller
// device arrays and builds no tdp_graph.  The only temporary storage it needs,
// one partial sum per block of 256 nets and a count of finished blocks, lives
// in a file-scope static device array of fixed size that is part of the
// library image: every GPU that loads the library holds it (128 KiB + 4 bytes)
// until the process exits.
#include <mutex>

#include "tdp_internal.cuh"

namespace tdp {
namespace {

constexpr int kNaThreads = 256;       // nets per block, one thread per net
constexpr int kNaMaxBlocks = 16384;   // partial-sum slots: at most 4,194,304 nets
constexpr int kNaMaxDevices = 64;

// Scratch shared by every call on a device: block partial sums and the count
// of finished blocks.  It keeps the last call's contents; the count is
// cleared before each launch.
static __device__ __align__(256) double g_na_part[kNaMaxBlocks];
static __device__ __align__(256) unsigned g_na_done[1];

struct NaScratch {
    double *part = nullptr;
    unsigned *done = nullptr;
    bool ready = false;
};
std::mutex g_na_mutex;
NaScratch g_na[kNaMaxDevices];

// One thread per net: beta-free sum of w_s ((x_s - x_d)^2 + (y_s - y_d)^2)
// over the net's sinks with a nonzero weight, FP32 terms, FP64 sums.  Each
// block leaves its sum in part[block]; the last block to finish adds the
// partials in block order, so the result does not depend on scheduling.
__global__ void __launch_bounds__(kNaThreads)
k_pp_fwd_noalloc(int n_nets, const int32_t *__restrict__ net_ptr, const int32_t *__restrict__ pin_cell,
                 const float *__restrict__ dx, const float *__restrict__ dy, const float *__restrict__ w,
                 const float *__restrict__ x, const float *__restrict__ y, double beta, double *loss,
                 double *part, unsigned *done) {
    __shared__ double sh[kNaThreads / 32];
    __shared__ bool last;
    const int e = blockIdx.x * kNaThreads + threadIdx.x;
    double acc = 0.0;
    const int a = e < n_nets ? net_ptr[e] : 0, b = e < n_nets ? net_ptr[e + 1] : 0;
    if (b > a) {  // an empty net (a caller error) adds nothing and reads no pin
        const int cd = pin_cell[a];
        const float xd = x[cd] + dx[a], yd = y[cd] + dy[a];
        for (int p = a + 1; p < b; ++p) {
            const float wp = w[p];
            if (wp == 0.0f) continue;
            const int cs = pin_cell[p];
            const float ux = x[cs] + dx[p] - xd, uy = y[cs] + dy[p] - yd;
            acc += (double)(wp * (ux * ux + uy * uy));
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < kNaThreads / 32; ++k) s += sh[k];
        part[blockIdx.x] = s;
        __threadfence();
        last = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x < 32) {
        __threadfence();
        const volatile double *vp = part;
        double v = 0.0;
        for (int k = threadIdx.x; k < (int)gridDim.x; k += 32) v += vp[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) *loss = beta * v;
    }
}

// Device addresses of the scratch for the current device, looked up once per
// device (with that device current) and kept.
tdp_status na_scratch(NaScratch *&out) {
    int dev = 0;
    TDP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNaMaxDevices) {
        set_error("attraction_loss_fwd_noalloc: device ordinal %d is not supported", dev);
        return TDP_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lock(g_na_mutex);
    NaScratch &s = g_na[dev];
    if (!s.ready) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_na_part);
        if (e != cudaSuccess) {
            set_error("attraction_loss_fwd_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return TDP_ERR_CUDA;
        }
        s.part = static_cast<double *>(p);
        e = cudaGetSymbolAddress(&p, g_na_done);
        if (e != cudaSuccess) {
            set_error("attraction_loss_fwd_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return TDP_ERR_CUDA;
        }
        s.done = static_cast<unsigned *>(p);
        s.ready = true;
    }
    out = &s;
    return TDP_OK;
}

}  // namespace
}  // namespace tdp

using namespace tdp;

extern "C" tdp_status attraction_loss_fwd_noalloc(int32_t n_nets, const int32_t *net_ptr_dev,
                                                  const int32_t *pin_cell_dev, const float *pin_dx_dev,
                                                  const float *pin_dy_dev, const float *w_dev,
                                                  const float *x_dev, const float *y_dev, double beta,
                                                  double *loss_dev, void *cuda_stream) {
    const int64_t max_nets = (int64_t)kNaThreads * kNaMaxBlocks;
    if (n_nets < 0 || !loss_dev || !std::isfinite(beta) ||
        (n_nets > 0 && (!net_ptr_dev || !pin_cell_dev || !pin_dx_dev || !pin_dy_dev || !w_dev || !x_dev ||
                        !y_dev))) {
        set_error("attraction_loss_fwd_noalloc: negative n_nets, NULL array or non-finite beta");
        return TDP_ERR_INVALID;
    }
    if (n_nets > max_nets) {
        set_error("attraction_loss_fwd_noalloc: %d nets exceed the static scratch, which holds at most "
                  "%lld nets (one partial sum per %d nets); use attraction_loss_fwd", n_nets,
                  (long long)max_nets, kNaThreads);
        return TDP_ERR_INVALID;
    }
    NaScratch *sc = nullptr;
    TDP_TRY(na_scratch(sc));
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (n_nets == 0) {
        TDP_CUDA(cudaMemsetAsync(loss_dev, 0, sizeof(double), st));
        return TDP_OK;
    }
    TDP_CUDA(cudaMemsetAsync(sc->done, 0, sizeof(unsigned), st));  // the count must start at zero
    k_pp_fwd_noalloc<<<div_up(n_nets, kNaThreads), kNaThreads, 0, st>>>(
        n_nets, net_ptr_dev, pin_cell_dev, pin_dx_dev, pin_dy_dev, w_dev, x_dev, y_dev, beta, loss_dev,
        sc->part, sc->done);
    TDP_LAUNCH_CHECK();
    return TDP_OK;
}
