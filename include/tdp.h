/*
 * tdp.h -- C ABI of the B300 timing hot path for path-based timing-driven
 * global placement ("Timing-Driven Global Placement by Efficient Critical
 * Path Extraction", arXiv 2503.11674).
 *
 * One timing iteration is
 *   sta_propagate            Section II-B, Eqs. (2)-(4), Eq. (8)
 *   extract_critical_paths   Section III-B, report_timing_endpoint(n, k)
 *   attraction_update_pairs  Section III-D, Eq. (w_ij)
 *   attraction_loss_fwd/bwd  Eq. (9) and the PP sum of Section III-D
 * and report_timing (Section III-B, Table I) is the global extraction that
 * report_timing_endpoint is compared against.
 *
 * Conventions shared by every entry point:
 *  - All pointers are plain C pointers.  "_dev" arguments are CUDA device
 *    pointers on the current device; "_host" / "_out" arguments are host
 *    pointers.  No PyTorch or C++ type crosses this boundary.
 *  - Floating-point device arrays ("void*") hold float for a graph built
 *    with TDP_FP32 and double for TDP_FP64.  Units: um, fF, kOhm, ps.
 *  - The caller owns every array it passes; the library only reads (or, for
 *    outputs, writes) them during the call, in stream order.  The library
 *    owns the graph, the timing arrays, the extracted paths and the pin-pair
 *    set P with its weights; it frees them in sta_destroy.
 *  - Work is queued on the CUDA stream given to sta_build.  A call returns
 *    after queueing, except where a non-NULL host "_out" pointer asks for a
 *    result, in which case it synchronises that stream first.
 *  - Every call returns a tdp_status.  Nothing throws or aborts across the
 *    boundary.  On a non-OK status tdp_last_error() describes the failure.
 *    Calls made out of order return TDP_ERR_STATE and change nothing.
 *  - A graph is not thread safe: one host thread at a time per graph.
 */
#ifndef TDP_H
#define TDP_H

#include <stdint.h>

#if defined(__GNUC__)
#define TDP_API __attribute__((visibility("default")))
#else
#define TDP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tdp_graph tdp_graph;

typedef enum {
    TDP_OK = 0,
    TDP_ERR_INVALID = 1,  /* bad argument or malformed netlist                 */
    TDP_ERR_CYCLE = 2,    /* combinational loop in the netlist                  */
    TDP_ERR_OOM = 3,      /* device or host allocation failed                   */
    TDP_ERR_CUDA = 4,     /* a CUDA runtime call or kernel launch failed        */
    TDP_ERR_STATE = 5,    /* call out of order (e.g. extract before propagate)  */
    TDP_ERR_TIMEOUT = 6   /* a level sweep's grid-wide wait gave up (bounded);
                             the results of that call are not valid           */
} tdp_status;

typedef enum { TDP_FP32 = 0, TDP_FP64 = 1 } tdp_precision;

/* pin-pair distance term of the attraction loss */
typedef enum {
    TDP_LOSS_QUADRATIC = 0, /* Q(i,j) = dx^2 + dy^2, Eq. (9) (default)          */
    TDP_LOSS_HPWL = 1,      /* |dx| + |dy|       (ablation, Section IV)          */
    TDP_LOSS_EUCLID = 2     /* sqrt(dx^2 + dy^2) (ablation, Section IV)          */
} tdp_loss_kind;

/* cell_type values */
enum { TDP_CELL_COMB = 0, TDP_CELL_FF = 1, TDP_CELL_PI = 2, TDP_CELL_PO = 3 };

/*
 * Netlist description (host arrays, read during sta_build only).
 *
 * Pins are numbered net-contiguously: net e owns pins net_ptr[e] ..
 * net_ptr[e+1]-1 and its first pin is the driver (pin_dir 1); every other pin
 * of the net is a sink (pin_dir 0).  Every pin belongs to exactly one net and
 * every net has at least one sink.
 *
 * Cell types and their pins:
 *   TDP_CELL_COMB  1..32 input pins and exactly one output pin;
 *   TDP_CELL_FF    at most one input (D, an endpoint) and at most one output
 *                  (Q, a startpoint);
 *   TDP_CELL_PI    primary input port: one output (startpoint), no input;
 *   TDP_CELL_PO    primary output port: one input (endpoint), no output.
 *
 * Delay model (Eq. (8) with R and C linear in wire length): the wire from a
 * net's driver to sink s has Manhattan length L between the pin positions
 * (cell position plus pin offset), Elmore delay
 *   t_s = r L (c L / 2 + pin_cap[s]),
 * and the net's load is C_load = sum over sinks of (c L + pin_cap[s]).  The
 * driving cell's delay d = d0 + cell_rdrv * C_load applies to every input
 * arc of a combinational cell, and is the launch (clock-to-Q) delay of a
 * flip-flop or primary input.  Single corner, late only, ideal clock at
 * t = 0, setup time 0.
 */
typedef struct {
    int32_t n_cells, n_pins, n_nets;
    const int32_t *pin_cell;   /* [n_pins]   owning cell of every pin           */
    const int32_t *net_ptr;    /* [n_nets+1] CSR of pins by net, driver first    */
    const uint8_t *pin_dir;    /* [n_pins]   1 driver, 0 sink                    */
    const int32_t *cell_type;  /* [n_cells]  TDP_CELL_*                          */
    const float *pin_dx;       /* [n_pins]   pin offset from the cell, um        */
    const float *pin_dy;       /* [n_pins]                                       */
    const float *pin_cap;      /* [n_pins]   fF (sinks; ignored on drivers)      */
    const float *cell_rdrv;    /* [n_cells]  drive resistance, kOhm              */
    const uint8_t *cell_fixed; /* [n_cells]  1: the cell gets zero gradient      */
    double r_per_um;           /* wire resistance, kOhm/um                       */
    double c_per_um;           /* wire capacitance, fF/um                        */
    double d0_ps;              /* intrinsic cell delay, ps                       */
} tdp_netlist_desc;

/*
 * Build the device timing graph (Section II-B): validate the netlist,
 * levelize the combinational cells, lay the CSR-by-level arrays out in device
 * memory and allocate all timing state for the given precision.
 * cuda_stream is a cudaStream_t (NULL = legacy default stream); all later
 * work of this graph is queued on it.
 * Errors: TDP_ERR_INVALID (malformed description), TDP_ERR_CYCLE
 * (combinational loop), TDP_ERR_OOM, TDP_ERR_CUDA.  *out is NULL on error.
 */
TDP_API tdp_status sta_build(const tdp_netlist_desc *netlist, tdp_precision precision, void *cuda_stream,
                     tdp_graph **out);

/* Free every device and host resource of the graph (NULL is a no-op). */
TDP_API void sta_destroy(tdp_graph *g);

/*
 * Static timing analysis at placement (x, y) (Section II-B; Eq. (2)
 * slack; Eqs. (3)-(4) WNS / TNS; Eq. (8) net delay).
 * x_dev, y_dev: [n_cells] cell positions (float or double by precision).
 * Computes Elmore net delays and cell delays, arrival times forward and
 * required times backward over the levels, the slack of every pin (of the
 * pins that are not endpoints when sta_get_timing asks for it), and
 * WNS = min slack over violated endpoints, TNS = sum of their slacks (both
 * 0 when no endpoint violates), reduced in FP64.
 * Endpoint slacks, WNS and TNS need the forward sweep only; path extraction,
 * the pair update and the loss read nothing else of the backward sweep.  So
 * the library runs the backward sweep (required times) on a second stream
 * of its own, beside whatever the caller queues next.  Calls that read its
 * results (sta_get_timing) or rewrite its inputs (the next sta_propagate)
 * make the graph's stream wait for it first; sta_join does the same on
 * request, e.g. before an event that times a whole iteration.  The
 * environment variable TDP_SERIAL_BWD=1 at sta_build keeps the backward
 * sweep on the graph's stream, in order.
 * wns_out / tns_out: host doubles, or NULL to skip the synchronisation.
 */
TDP_API tdp_status sta_propagate(tdp_graph *g, const void *x_dev, const void *y_dev,
                         double clock_period_ps, double *wns_out, double *tns_out);

/*
 * Incremental timing: the same results as sta_propagate, bit for bit, for
 * positions that differ from those of the graph's last propagation in a
 * few cells only.  Section IV re-times the design every m placement steps;
 * between two such points few cells may have moved (or, in a loop that
 * moves cells one at a time, one).  The call compares x_dev / y_dev with the
 * positions of the last propagation (bit for bit) and re-times:
 *   - the nets with a pin on a moved cell (Eq. (8): Elmore delays, load,
 *     delay of the driving cell), each counted as changed;
 *   - in the forward sweep, only the cells with a changed input or delay,
 *     over the levels the changes reach; a re-evaluated cell whose arrival,
 *     worst input, chain length and sidetrack list come out unchanged stops
 *     the change there.  Once a level's changed cells exceed 1/16 of the
 *     next level's cells, every later cell is evaluated without checks
 *     (changes spread through the sidetrack lists to most cells downstream);
 *   - the endpoints, WNS / TNS and the backward sweep in full (the backward
 *     sweep runs beside later calls, as in sta_propagate).
 * Arguments, outputs, stream order and errors as for sta_propagate.  The
 * first call on a graph, and any call after which the previous state cannot
 * serve (no earlier propagation, a failed one, per-level launches instead of
 * a single launch), re-times everything.  From the first call on, the graph
 * keeps the positions of every propagation (sta_propagate too): 2 * n_cells
 * floats or doubles, plus 16 bytes per net.
 */
TDP_API tdp_status sta_propagate_incremental(tdp_graph *g, const void *x_dev, const void *y_dev,
                                             double clock_period_ps, double *wns_out, double *tns_out);

/*
 * What the last propagation re-timed (synchronises the graph's stream).
 * stats_out: host int64_t[7]:
 *   [0] 1 if it re-timed everything (sta_propagate, or a first or fallback
 *       sta_propagate_incremental; then [1]..[5] count every cell and
 *       level), else 0
 *   [1] cells that moved
 *   [2] combinational cells re-evaluated selectively (an input or the
 *       cell's delay changed) in the forward sweep
 *   [3] of them, cells whose outputs changed
 *   [4], [5] first and last level of the forward sweep (0, -1: none)
 *   [6] level from which the sweep evaluated every cell, without checks
 *       (0: none): once the changed cells of a level exceed 1/16 of the
 *       next level's cells, checking costs more than it saves
 * Errors: TDP_ERR_STATE before the first propagation.
 */
TDP_API tdp_status sta_incremental_stats(tdp_graph *g, int64_t *stats_out);

/*
 * Make the graph's stream wait for the backward sweep of the last
 * sta_propagate (queued on the library's second stream).  No-op if nothing
 * is outstanding.  Does not synchronise the host.
 */
TDP_API tdp_status sta_join(tdp_graph *g);

/*
 * Copy per-pin arrival, required time and slack (float/double [n_pins]) of the
 * last sta_propagate into caller device buffers; any pointer may be NULL.
 * Errors: TDP_ERR_STATE before the first sta_propagate.
 */
TDP_API tdp_status sta_get_timing(tdp_graph *g, void *arr_dev, void *req_dev, void *slack_dev);

/*
 * Copy the net delays of the last sta_propagate: Elmore delay of every pin
 * (0 on drivers) [n_pins], and per net the load C_load and the delay d of its
 * driving cell [n_nets] (Eq. (8)).  Any pointer may be NULL.
 */
TDP_API tdp_status sta_get_net_delays(tdp_graph *g, void *tnet_dev, void *cload_dev, void *dcell_dev);

/*
 * report_timing_endpoint(n, K) (Section III-B): sort the failing endpoints
 * by (slack, pin) ascending, take the n most critical (n < 0: all of them),
 * and extract for each its K lowest-slack startpoint-to-endpoint paths
 * (rank 1 is the worst path).  With keep_nonneg == 0 only paths of negative
 * slack are kept, so an endpoint may return fewer than K; with
 * keep_nonneg != 0 up to K paths are kept whatever their slack.  Equal-slack
 * paths are ordered by their pin sequences read from the endpoint
 * backwards (lexicographic, smaller first); argmax ties take the lowest pin.
 * 1 <= K <= 32.  n_paths_out: host int64 or NULL (no synchronisation).
 * The paths stay valid until the next extract_critical_paths or
 * sta_propagate.  Errors: TDP_ERR_STATE before sta_propagate.
 */
TDP_API tdp_status extract_critical_paths(tdp_graph *g, int32_t n_endpoints, int32_t K,
                                  int32_t keep_nonneg, int64_t *n_paths_out);

/*
 * report_timing(n) (Section III-B, Table I; OpenTimer's semantics): the n
 * worst endpoints, the n worst paths of each, and of those n^2 paths the n
 * of lowest slack -- which are the n lowest-slack startpoint-to-endpoint
 * paths of the whole design.  With keep_nonneg == 0 only paths of negative
 * slack are reported (fewer than n when the design has fewer); with
 * keep_nonneg != 0 every endpoint takes part whatever its slack.  The
 * paths are reported worst first; equal-slack paths are ordered
 * deterministically by the search, not by pin sequence.  n >= 0 (n = 0:
 * no path).  The search holds one record per candidate path; its memory
 * grows with n and with the number of near-critical paths of the design.
 * It replaces the last extraction: sta_get_paths_size / sta_get_paths
 * return these paths (viol_dev: the failing endpoints, as for
 * extract_critical_paths) and attraction_update_pairs takes them as its
 * path set.  The paths stay valid until the next extraction or
 * sta_propagate.  The search reads its sizes back between rounds, so this
 * call synchronises the stream.  n_paths_out: host int64 or NULL.
 * Errors: TDP_ERR_INVALID for n < 0; TDP_ERR_STATE before sta_propagate;
 * TDP_ERR_OOM when the search needs more than 2^31 - 1 path records or
 * the device memory for them.
 */
TDP_API tdp_status report_timing(tdp_graph *g, int32_t n, int32_t keep_nonneg, int64_t *n_paths_out);

/*
 * Sizes of the last extraction (synchronises): number of failing endpoints,
 * number of paths, total number of pins over all paths.
 */
TDP_API tdp_status sta_get_paths_size(tdp_graph *g, int32_t *n_viol_out, int64_t *n_paths_out,
                              int64_t *n_path_pins_out);

/*
 * Materialise the extracted paths into caller device buffers, endpoints in
 * (slack, pin) order and paths by rank within an endpoint:
 *   viol_dev    int32[n_viol]      failing endpoints, most critical first;
 *   ep_dev      int32[n_paths]     endpoint pin of every path;
 *   slack_dev   float/double[n_paths] path slack (T - path delay);
 *   pin_ptr_dev int64[n_paths+1]   offsets into pins_dev;
 *   pins_dev    int32[n_path_pins] pins of each path, startpoint first.
 * Any pointer may be NULL.  Sizes come from sta_get_paths_size.
 */
TDP_API tdp_status sta_get_paths(tdp_graph *g, int32_t *viol_dev, int32_t *ep_dev, void *slack_dev,
                         int64_t *pin_ptr_dev, int32_t *pins_dev);

/*
 * Eq. (w_ij) (Section III-D): traverse the extracted paths, worst first.
 * Every net arc (driver -> sink s) on a path is a pin pair, identified by s.
 * A pair not yet in P enters P with weight w0; a pair already in P gains
 * w1 * slack / WNS, slack being the path's slack and WNS the last
 * sta_propagate's.  Contributions of all paths through a pair add up
 * (path sharing); the result does not depend on the order of the paths.
 * P and the weights persist across calls until attraction_reset_pairs.
 * n_pairs_out: host int64 (|P| after the update) or NULL.
 * Errors: TDP_ERR_STATE before extract_critical_paths.
 */
TDP_API tdp_status attraction_update_pairs(tdp_graph *g, double w0, double w1, int64_t *n_pairs_out);

/* Empty the pin-pair set P. */
TDP_API tdp_status attraction_reset_pairs(tdp_graph *g);

/*
 * Replace P by the n_pairs sink pins in pins_host (each a sink pin, no
 * duplicates) with weights w_host (host arrays, read during the call).
 * Used to restore a saved state.  Errors: TDP_ERR_INVALID.
 */
TDP_API tdp_status attraction_set_pairs(tdp_graph *g, int64_t n_pairs, const int32_t *pins_host,
                                const double *w_host);

/*
 * Copy P into caller device buffers: pins_dev int32[|P|] (sink pins,
 * ascending) and w_dev float/double[|P|]; n_pairs_out (host) receives |P|
 * (synchronises).  Either buffer may be NULL to query the size only.
 */
TDP_API tdp_status attraction_get_pairs(tdp_graph *g, int32_t *pins_dev, void *w_dev,
                                int64_t *n_pairs_out);

/*
 * Pin-to-pin attraction loss (Eq. (9) and PP of Section III-D):
 *   loss = beta * sum over (driver, s) in P of w_s * Q(driver, s),
 *   Q(i, j) = (x_i - x_j)^2 + (y_i - y_j)^2 on pin coordinates.
 * x_dev, y_dev: [n_cells]; loss_dev: one device double (overwritten).
 * Terms in the graph's precision, the total in FP64; deterministic.
 */
TDP_API tdp_status attraction_loss_fwd(tdp_graph *g, const void *x_dev, const void *y_dev, double beta,
                               double *loss_dev);

/*
 * Adjoint of attraction_loss_fwd: gx_dev, gy_dev [n_cells] are overwritten
 * with grad_scale * dloss/dx, dloss/dy, where grad_scale is the device
 * double *grad_scale_dev (NULL means 1).  Per sink s in P the pin gradient is
 * 2 beta w_s (p_s - p_driver); the driver receives minus the sum over its
 * sinks; a cell receives the sum of its pins' gradients, accumulated in FP64
 * in a fixed order (no floating-point atomics); fixed cells receive 0.
 */
TDP_API tdp_status attraction_loss_bwd(tdp_graph *g, const void *x_dev, const void *y_dev, double beta,
                               const double *grad_scale_dev, void *gx_dev, void *gy_dev);

/*
 * attraction_loss_fwd_bwd: attraction_loss_fwd and attraction_loss_bwd in one
 * call, for callers that need the loss and its gradient every step (a
 * placer's step; the paper adds beta PP to the placement objective, Section
 * III-A): the same loss and gradient, bit for bit, in two launches instead
 * of three (the per-pair pass computes the terms with the pin gradients).
 * Arguments as the two calls: x_dev, y_dev positions; beta; grad_scale_dev a
 * device double scaling the gradient (NULL: 1); loss_dev one device double;
 * gx_dev, gy_dev overwritten.  Stream-ordered, no host synchronisation.
 * Errors: TDP_ERR_INVALID (NULL graph or argument, non-finite beta),
 * TDP_ERR_CUDA.
 */
TDP_API tdp_status attraction_loss_fwd_bwd(tdp_graph *g, const void *x_dev, const void *y_dev, double beta,
                                           const double *grad_scale_dev, double *loss_dev, void *gx_dev,
                                           void *gy_dev);

/*
 * attraction_set_loss_kind: the pair term Q(i, j) of later
 * attraction_loss_fwd / _bwd calls on g.  TDP_LOSS_QUADRATIC (the default)
 * is Eq. (9).  TDP_LOSS_HPWL (|dx| + |dy|, pin gradient beta w_s sign(dx),
 * sign(dy), 0 at 0) and TDP_LOSS_EUCLID (sqrt(dx^2 + dy^2), pin gradient
 * beta w_s (dx, dy) / d, 0 when the pins coincide) are the alternatives the
 * ablation of Section IV compares; the paper names them without formulas.
 * Errors: TDP_ERR_INVALID (NULL graph, unknown kind).
 */
TDP_API tdp_status attraction_set_loss_kind(tdp_graph *g, tdp_loss_kind kind);

/*
 * Net weighting from pin slacks, with momentum: the net-weighting scheme the
 * paper compares its pin-pair attraction against (Section II-C, the weighted
 * wirelength objective sum_e w_e WL_e; the "w/o Path Extraction" column of
 * the ablation, Section IV, DREAMPlace 4.0's pin-level scheme).  The paper
 * names the scheme without its formula; this library reads it as
 *   s_e  = the worst slack over the pins of net e (equal to its driver
 *          pin's slack, as sta_get_timing reports it),
 *   c_e  = min(1, max(0, -s_e) / |WNS|)  (0 when WNS = 0),
 *   w_e <- alpha * w_e + (1 - alpha) * (1 + gamma * c_e),
 * with every w_e starting at 1 (sta_build, net_weights_reset).  The weights
 * are for the caller's weighted wirelength; this library computes no
 * wirelength.
 * net_weights_update: one update from the last sta_propagate (waits for its
 *   backward sweep).  alpha in [0, 1] (momentum), gamma >= 0 (weight gain).
 *   n_critical_out: host int64, the number of nets with s_e < 0 (the call
 *   then synchronises), or NULL.  Stream-ordered otherwise.
 * net_weights_get: copies the weights (float or double [n_nets], the graph's
 *   precision) to w_dev; stream-ordered.
 * net_weights_reset: every weight back to 1.
 * Errors: TDP_ERR_INVALID (NULL graph or output, alpha or gamma out of
 * range), TDP_ERR_STATE (update before sta_propagate), TDP_ERR_OOM,
 * TDP_ERR_CUDA, TDP_ERR_TIMEOUT (as sta_propagate).
 */
TDP_API tdp_status net_weights_update(tdp_graph *g, double alpha, double gamma, int64_t *n_critical_out);
TDP_API tdp_status net_weights_get(tdp_graph *g, void *w_dev);
TDP_API tdp_status net_weights_reset(tdp_graph *g);

/*
 * attraction_loss_fwd for callers that cannot allocate device memory (no
 * counterpart in the paper): code working inside a device-memory budget fixed
 * in advance, code whose allocator owns all device memory, or code that must
 * not allocate after start-up cannot call sta_build, which allocates.  This
 * entry point needs no tdp_graph and calls no cudaMalloc, cudaFree or other
 * allocating routine: every input and the output are caller device arrays,
 * and its temporary storage (one FP64 partial sum per 256 nets and a block
 * counter) is a static device array of the library, 128 KiB + 4 bytes held
 * on every GPU that loads the library until the process exits.
 *   n_nets        nets; at most 4,194,304 (more: TDP_ERR_INVALID)
 *   net_ptr_dev   int32[n_nets+1] pins of each net, driver first (as sta_build):
 *                 non-decreasing, net_ptr[0] = 0; every net should hold its
 *                 driver pin and at least one sink (sta_build rejects other
 *                 nets; here an empty net adds nothing and reads no pin).
 *                 This call does not validate the arrays: they are not
 *                 read on the host
 *   pin_cell_dev  int32[n_pins], pin_dx_dev / pin_dy_dev float[n_pins] (um)
 *   w_dev         float[n_pins] weight of the pair (driver, pin) of every sink
 *                 pin; 0 for pins not in P (and ignored on drivers)
 *   x_dev, y_dev  float[n_cells] cell positions
 *   loss_dev      one device double, overwritten with
 *                 beta * sum over sinks s with w_s != 0 of w_s * Q(driver, s)
 *   cuda_stream   cudaStream_t the work is queued on (NULL: legacy stream)
 * FP32 terms, FP64 sums, fixed-order reduction (deterministic).  The first
 * call on a device looks up the scratch address for that device (with it
 * current); make that first call before capturing any stream into a CUDA
 * graph.  All calls on a device share the scratch: calls that overlap on the
 * GPU (other streams, or graph replays running at once) race and give wrong
 * results; calls queued on one stream are safe.
 */
TDP_API tdp_status attraction_loss_fwd_noalloc(int32_t n_nets, const int32_t *net_ptr_dev,
                                               const int32_t *pin_cell_dev, const float *pin_dx_dev,
                                               const float *pin_dy_dev, const float *w_dev,
                                               const float *x_dev, const float *y_dev, double beta,
                                               double *loss_dev, void *cuda_stream);

/*
 * Instrumentation (no counterpart in the paper).
 * tdp_get_launch_count: number of kernels this graph has queued so far
 * (graph replays count every kernel node).
 * tdp_profile_kernel: time every later launch of the named kernel with a pair
 * of CUDA events on the graph's stream: "net_rc", "fwd_sweep" (one replay of
 * the forward level kernels), "bwd_sweep" (the backward level kernels and
 * WNS / TNS), "viol_sort" (the whole endpoint sort), "topk", "pair_walk",
 * "pair_finish", "pp_fwd", "pp_bwd_net", "pp_bwd_cell", "rt_expand",
 * "ep_wns", "inc_moved", "fwd_inc", "net_weights", "pp_fwd_bwd"; NULL or "" stops.
 * tdp_profile_read: synchronise the stream, return the number of timed
 * launches and their summed device time in ms, and reset both.
 */
TDP_API tdp_status tdp_get_launch_count(tdp_graph *g, int64_t *n_out);
TDP_API tdp_status tdp_profile_kernel(tdp_graph *g, const char *kernel_name);
TDP_API tdp_status tdp_profile_read(tdp_graph *g, int64_t *launches_out, double *total_ms_out);

/*
 * tdp_selftest_grid_wait: test hook of the bounded grid-wide wait that the
 * single-launch level sweeps use between levels (the paper has no
 * counterpart).  Launches, on the current device and the legacy default
 * stream, a cooperative kernel of two blocks whose barrier waits for one
 * more arrival than there are blocks, so that the wait must give up after
 * timeout_ms; synchronises, and sets *gave_up_out to 1 if the kernel
 * recorded the timeout status, else 0.  Allocates and frees 8 bytes of
 * device memory.  Errors: TDP_ERR_INVALID (NULL output, timeout_ms not in
 * (0, 1000]), TDP_ERR_CUDA.
 */
TDP_API tdp_status tdp_selftest_grid_wait(double timeout_ms, int32_t *gave_up_out);

/*
 * Test hooks of the host-side failure paths (no counterpart in the paper).
 * They make a failure on the host; none of them faults, traps or stalls a
 * GPU.
 * tdp_debug_fail_alloc: the n-th next device allocation the library makes
 * (process-wide, any graph; cudaMalloc of graph state or cudaMallocAsync of
 * a temporary) fails as if the device were out of memory, without calling
 * CUDA; the call that made it returns TDP_ERR_OOM and frees what it had
 * allocated.  n = 0 cancels a pending failure.  Errors: TDP_ERR_INVALID
 * (n < 0).
 * tdp_debug_pending_alloc_failure: *n_out = the countdown left (0: none
 * pending, i.e. the injected failure has happened or was cancelled).
 * tdp_debug_set_sync_status: writes `status` into the graph's sticky status
 * word of the level sweeps' grid-wide waits (the word a wait that gave up
 * sets), on the graph's stream, and synchronises.  A non-zero status makes
 * the next host-synchronising call that checks the word (sta_propagate with
 * wns_out or tns_out, extract_critical_paths with n_paths_out,
 * report_timing) return TDP_ERR_TIMEOUT, clear the word and mark the timing
 * results invalid, as after a real timeout.  Errors: TDP_ERR_INVALID (NULL
 * graph), TDP_ERR_CUDA.
 */
TDP_API tdp_status tdp_debug_fail_alloc(int64_t n);
TDP_API tdp_status tdp_debug_pending_alloc_failure(int64_t *n_out);
TDP_API tdp_status tdp_debug_set_sync_status(tdp_graph *g, uint32_t status);

/* Message for the last non-OK status returned on this host thread. */
TDP_API const char *tdp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TDP_H */
