/*
 * A consumer of the library written in plain C (C99): it includes only
 * include/tdp.h and the CUDA runtime's C header, links the shared library,
 * and runs one timing iteration on the three-cell chain of
 * tests/golden/chain3.json (flip-flop A -> combinational B -> flip-flop C),
 * whose every value is derived there by hand from Eq. (8), Section II-B and
 * Eqs. (2)-(4), Section III-B, Eq. (w_ij) and Eq. (9).
 *
 * Exit status: 0 every result matches; 1 a call returned an error status;
 * 2 a result is off; 3 no CUDA device (the library is never called then).
 */
#include <math.h>
#include <stdio.h>
#include <stdint.h>

#include <cuda_runtime_api.h>

#include "tdp.h"

static int fails = 0;

static void expect(const char *what, double got, double want, double tol) {
    if (!(fabs(got - want) <= tol)) {
        printf("%s: %.9g, expected %.9g\n", what, got, want);
        ++fails;
    }
}

#define CALL(x)                                                                      \
    do {                                                                             \
        tdp_status st_ = (x);                                                        \
        if (st_ != TDP_OK) {                                                         \
            printf("%s -> status %d: %s\n", #x, (int)st_, tdp_last_error());        \
            return 1;                                                                \
        }                                                                            \
    } while (0)

int main(void) {
    int n_dev = 0;
    if (cudaGetDeviceCount(&n_dev) != cudaSuccess || n_dev == 0) {
        printf("no CUDA device\n");
        return 3;
    }
    /* pins: 0 A.Q (driver), 1 B.in, 2 B.out (driver), 3 C.D */
    const int32_t pin_cell[4] = {0, 1, 1, 2};
    const int32_t net_ptr[3] = {0, 2, 4};
    const uint8_t pin_dir[4] = {1, 0, 1, 0};
    const int32_t cell_type[3] = {TDP_CELL_FF, TDP_CELL_COMB, TDP_CELL_FF};
    const float pin_dx[4] = {0, 0, 0, 0}, pin_dy[4] = {0, 0, 0, 0};
    const float pin_cap[4] = {1.0f, 2.0f, 1.0f, 1.0f};
    const float cell_rdrv[3] = {1.0f, 2.0f, 1.0f};
    const uint8_t cell_fixed[3] = {0, 0, 0};
    tdp_netlist_desc d;
    d.n_cells = 3;
    d.n_pins = 4;
    d.n_nets = 2;
    d.pin_cell = pin_cell;
    d.net_ptr = net_ptr;
    d.pin_dir = pin_dir;
    d.cell_type = cell_type;
    d.pin_dx = pin_dx;
    d.pin_dy = pin_dy;
    d.pin_cap = pin_cap;
    d.cell_rdrv = cell_rdrv;
    d.cell_fixed = cell_fixed;
    d.r_per_um = 0.004;
    d.c_per_um = 0.2;
    d.d0_ps = 5.0;

    tdp_graph *g = NULL;
    CALL(sta_build(&d, TDP_FP32, NULL, &g));

    const float hx[3] = {0.0f, 100.0f, 100.0f}, hy[3] = {0.0f, 0.0f, 50.0f};
    float *x = NULL, *y = NULL, *gx = NULL, *gy = NULL, *slack = NULL, *w = NULL;
    double *loss = NULL;
    int32_t *ep = NULL, *pins = NULL, *ppins = NULL;
    int64_t *pin_ptr = NULL;
    if (cudaMalloc((void **)&x, sizeof hx) != cudaSuccess || cudaMalloc((void **)&y, sizeof hy) != cudaSuccess ||
        cudaMalloc((void **)&gx, sizeof hx) != cudaSuccess || cudaMalloc((void **)&gy, sizeof hy) != cudaSuccess ||
        cudaMalloc((void **)&loss, sizeof(double)) != cudaSuccess ||
        cudaMalloc((void **)&ep, 16 * sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc((void **)&slack, 16 * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void **)&pin_ptr, 17 * sizeof(int64_t)) != cudaSuccess ||
        cudaMalloc((void **)&pins, 64 * sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc((void **)&ppins, 16 * sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc((void **)&w, 16 * sizeof(float)) != cudaSuccess) {
        printf("cudaMalloc failed\n");
        return 1;
    }
    cudaMemcpy(x, hx, sizeof hx, cudaMemcpyHostToDevice);
    cudaMemcpy(y, hy, sizeof hy, cudaMemcpyHostToDevice);

    /* STA at T = 50 ps: arrival 60 ps at C.D, slack -10 ps on the whole path */
    double wns = 0.0, tns = 0.0;
    CALL(sta_propagate(g, x, y, 50.0, &wns, &tns));
    expect("WNS", wns, -10.0, 1e-3);
    expect("TNS", tns, -10.0, 1e-3);
    float arr[4], req[4], sl[4];
    float *arr_d = NULL, *req_d = NULL, *sl_d = NULL;
    cudaMalloc((void **)&arr_d, sizeof arr);
    cudaMalloc((void **)&req_d, sizeof req);
    cudaMalloc((void **)&sl_d, sizeof sl);
    CALL(sta_get_timing(g, arr_d, req_d, sl_d));
    cudaDeviceSynchronize();
    cudaMemcpy(arr, arr_d, sizeof arr, cudaMemcpyDeviceToHost);
    cudaMemcpy(req, req_d, sizeof req, cudaMemcpyDeviceToHost);
    cudaMemcpy(sl, sl_d, sizeof sl, cudaMemcpyDeviceToHost);
    const double arr_e[4] = {27.0, 31.8, 58.8, 60.0}, req_e[4] = {17.0, 21.8, 48.8, 50.0};
    for (int p = 0; p < 4; ++p) {
        expect("arrival", arr[p], arr_e[p], 1e-3);
        expect("required", req[p], req_e[p], 1e-3);
        expect("slack", sl[p], -10.0, 1e-3);
    }

    /* report_timing_endpoint(-1, 1): the one path A.Q -> B.in -> B.out -> C.D */
    int64_t n_paths = 0, n_pins = 0;
    int32_t n_viol = 0;
    CALL(extract_critical_paths(g, -1, 1, 0, &n_paths));
    CALL(sta_get_paths_size(g, &n_viol, &n_paths, &n_pins));
    if (n_viol != 1 || n_paths != 1 || n_pins != 4) {
        printf("paths: %d failing endpoints, %lld paths, %lld pins\n", n_viol, (long long)n_paths,
               (long long)n_pins);
        ++fails;
    } else {
        int32_t hp[4], hep = -1;
        float hsl = 0.0f;
        CALL(sta_get_paths(g, NULL, ep, slack, pin_ptr, pins));
        cudaDeviceSynchronize();
        cudaMemcpy(hp, pins, sizeof hp, cudaMemcpyDeviceToHost);
        cudaMemcpy(&hep, ep, sizeof hep, cudaMemcpyDeviceToHost);
        cudaMemcpy(&hsl, slack, sizeof hsl, cudaMemcpyDeviceToHost);
        for (int k = 0; k < 4; ++k) expect("path pin", hp[k], k, 0.0);
        expect("path endpoint", hep, 3, 0.0);
        expect("path slack", hsl, -10.0, 1e-3);
    }

    /* Eq. (w_ij) with w0 = 10, w1 = 0.2: the path's two net arcs enter P at w0 */
    int64_t n_pairs = 0;
    CALL(attraction_update_pairs(g, 10.0, 0.2, &n_pairs));
    expect("pairs", (double)n_pairs, 2.0, 0.0);
    if (n_pairs == 2) {
        int32_t hpp[2];
        float hw[2];
        CALL(attraction_get_pairs(g, ppins, w, &n_pairs));
        cudaMemcpy(hpp, ppins, sizeof hpp, cudaMemcpyDeviceToHost);
        cudaMemcpy(hw, w, sizeof hw, cudaMemcpyDeviceToHost);
        for (int k = 0; k < 2; ++k) {
            expect("pair pin", hpp[k], k == 0 ? 1 : 3, 0.0);
            expect("pair weight", hw[k], 10.0, 1e-5);
        }
    }

    /* Eq. (9), beta = 1: PP = 10 (100^2) + 10 (50^2) = 125000 and its gradient */
    double hl = 0.0;
    float hgx[3], hgy[3];
    CALL(attraction_loss_fwd(g, x, y, 1.0, loss));
    CALL(attraction_loss_bwd(g, x, y, 1.0, NULL, gx, gy));
    cudaDeviceSynchronize();
    cudaMemcpy(&hl, loss, sizeof hl, cudaMemcpyDeviceToHost);
    cudaMemcpy(hgx, gx, sizeof hgx, cudaMemcpyDeviceToHost);
    cudaMemcpy(hgy, gy, sizeof hgy, cudaMemcpyDeviceToHost);
    expect("loss", hl, 125000.0, 1e-2);
    const double gx_e[3] = {-2000.0, 2000.0, 0.0}, gy_e[3] = {0.0, -1000.0, 1000.0};
    for (int c = 0; c < 3; ++c) {
        expect("gx", hgx[c], gx_e[c], 1e-2);
        expect("gy", hgy[c], gy_e[c], 1e-2);
    }

    /* incremental timing at the same placement: the first call re-times
       everything, the second finds no cell moved; both give WNS = TNS = -10 */
    double iw = 0.0, it = 0.0;
    int64_t stats[7];
    CALL(sta_propagate_incremental(g, x, y, 50.0, &iw, &it));
    expect("incremental WNS (first call)", iw, -10.0, 1e-4);
    CALL(sta_propagate_incremental(g, x, y, 50.0, &iw, &it));
    CALL(sta_incremental_stats(g, stats));
    expect("incremental WNS", iw, -10.0, 1e-4);
    expect("incremental TNS", it, -10.0, 1e-4);
    expect("incremental call re-timed everything", (double)stats[0], 0.0, 0.0);
    expect("moved cells", (double)stats[1], 0.0, 0.0);
    expect("cells re-evaluated", (double)stats[2], 0.0, 0.0);

    sta_destroy(g);
    cudaFree(x);
    cudaFree(y);
    cudaFree(gx);
    cudaFree(gy);
    cudaFree(loss);
    cudaFree(ep);
    cudaFree(slack);
    cudaFree(pin_ptr);
    cudaFree(pins);
    cudaFree(ppins);
    cudaFree(w);
    cudaFree(arr_d);
    cudaFree(req_d);
    cudaFree(sl_d);
    if (fails) return 2;
    printf("chain3 through the C ABI: all results match\n");
    return 0;
}
