/*
 * FP64 CPU oracle for the per-timing-iteration hot path of
 * "Timing-Driven Global Placement by Efficient Critical Path Extraction"
 * (arXiv 2503.11674).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference that the CUDA library is checked against.  It shares no code,
 * header, table or helper with the CUDA library; only tests, the smoke entry
 * point and the benchmark's CPU-baseline leg may load it.
 *
 * Everything is plain single-threaded C in double precision, written from the
 * paper's definitions:
 *   or_sta          Section II-B (timing graph, Arr forward / Req backward),
 *                   Eq. (2) slack, Eqs. (3)-(4) WNS/TNS, Eq. (8) RC net delay.
 *   or_topk         Section III-B, report_timing_endpoint(n, k): the k worst
 *                   paths of each of the n most critical failing endpoints,
 *                   found by a best-first search whose bound is the exact
 *                   arrival time.
 *   or_update_pairs Section III-D, Eq. (w_ij): the literal traversal of the
 *                   extracted paths, worst path first.
 *   or_loss         Eq. (9) quadratic pin-to-pin loss Q(i,j), and the PP sum
 *                   of Section III-D, with its analytic gradient;
 *                   or_loss_kind also the HPWL and linear Euclidean pair
 *                   distances of the ablation (Section IV).
 *   or_net_weights  the net-weighting baseline (Section II-C; the "w/o Path
 *                   Extraction" ablation of Section IV): net weights from
 *                   the worst pin slack on each net, with momentum (a stated
 *                   reading: the paper gives no formula).
 *
 * Where the paper is silent (delay model, ties, endpoints) this file reads
 * it as follows: single corner, late only, ideal clock
 * at t = 0, setup time 0; cell delay d = d0 + R_drv * C_load applies to every
 * input arc of the cell and is the clock-to-Q / launch delay of flip-flops and
 * primary inputs; argmax ties go to the lowest pin index; equal-slack paths
 * are ordered by their pin sequences read from the endpoint backwards.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { COMB = 0, FF = 1, PI = 2, PO = 3 };
enum { OR_OK = 0, OR_ERR_CYCLE = 2, OR_ERR_OOM = 3, OR_ERR_INVALID = 1 };

/* ------------------------------------------------------------------------ */
/* Netlist helpers                                                           */
/* ------------------------------------------------------------------------ */

typedef struct {
    int n_cells, n_pins, n_nets;
    const int32_t *pin_cell, *net_ptr, *cell_type;
    int32_t *pin_net;      /* net of every pin                              */
    int32_t *cp_ptr, *cp;  /* cell -> its pins, ascending pin index         */
} nl_t;

static int nl_init(nl_t *nl, int n_cells, int n_pins, int n_nets, const int32_t *pin_cell,
                   const int32_t *net_ptr, const int32_t *cell_type) {
    nl->n_cells = n_cells; nl->n_pins = n_pins; nl->n_nets = n_nets;
    nl->pin_cell = pin_cell; nl->net_ptr = net_ptr; nl->cell_type = cell_type;
    nl->pin_net = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_pins > 0 ? n_pins : 1));
    nl->cp_ptr = (int32_t *)calloc((size_t)n_cells + 1, sizeof(int32_t));
    nl->cp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_pins > 0 ? n_pins : 1));
    if (!nl->pin_net || !nl->cp_ptr || !nl->cp) return OR_ERR_OOM;
    for (int e = 0; e < n_nets; ++e)
        for (int p = net_ptr[e]; p < net_ptr[e + 1]; ++p) nl->pin_net[p] = e;
    for (int p = 0; p < n_pins; ++p) nl->cp_ptr[pin_cell[p] + 1]++;
    for (int c = 0; c < n_cells; ++c) nl->cp_ptr[c + 1] += nl->cp_ptr[c];
    int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n_cells + 1));
    if (!fill) return OR_ERR_OOM;
    memcpy(fill, nl->cp_ptr, sizeof(int32_t) * ((size_t)n_cells + 1));
    for (int p = 0; p < n_pins; ++p) nl->cp[fill[pin_cell[p]]++] = p;
    free(fill);
    return OR_OK;
}

static void nl_free(nl_t *nl) {
    free(nl->pin_net); free(nl->cp_ptr); free(nl->cp);
}

static int is_driver(const nl_t *nl, int p) { return nl->net_ptr[nl->pin_net[p]] == p; }

/* A startpoint is the output pin of a flip-flop (Q) or of a primary input. */
static int is_startpoint(const nl_t *nl, int p) {
    int t = nl->cell_type[nl->pin_cell[p]];
    return is_driver(nl, p) && (t == FF || t == PI);
}

/* An endpoint is the input pin of a flip-flop (D) or of a primary output. */
static int is_endpoint(const nl_t *nl, int p) {
    int t = nl->cell_type[nl->pin_cell[p]];
    return !is_driver(nl, p) && (t == FF || t == PO);
}

/* The output (driver) pin of a combinational cell, or -1. */
static int comb_output(const nl_t *nl, int cell) {
    for (int k = nl->cp_ptr[cell]; k < nl->cp_ptr[cell + 1]; ++k)
        if (is_driver(nl, nl->cp[k])) return nl->cp[k];
    return -1;
}

/* ------------------------------------------------------------------------ */
/* Static timing analysis (Section II-B, Eqs. (2)-(4), Eq. (8))             */
/* ------------------------------------------------------------------------ */

/*
 * Timing graph on pins.  Arcs:
 *   net arc  driver(e) -> sink s of e,  delay tnet[s]  (Elmore, Eq. (8));
 *   cell arc input i of a combinational cell -> its output o, delay dnet[net(o)].
 * Startpoints (FF Q, PI) have Arr = d of their cell (launch at t = 0);
 * endpoints (FF D, PO) have Req = T.
 */
int or_sta(int n_cells, int n_pins, int n_nets, const int32_t *pin_cell, const int32_t *net_ptr,
           const int32_t *cell_type, const double *pin_dx, const double *pin_dy,
           const double *pin_cap, const double *cell_rdrv, double r, double c, double d0,
           const double *x, const double *y, double T, double *tnet, double *cload,
           double *dnet, double *arr, double *req, double *slack, int32_t *pred, double *wns,
           double *tns) {
    nl_t nl;
    int st = nl_init(&nl, n_cells, n_pins, n_nets, pin_cell, net_ptr, cell_type);
    if (st) { nl_free(&nl); return st; }

    /* Eq. (8) with R and C linear in the Manhattan length L between the pins:
     * R = r L, and the wire capacitance c L is distributed along the wire, so
     * the Elmore delay to a sink of capacitance C_pin is r L (c L / 2 + C_pin).
     * The load seen by the driver is the sum of wire and pin capacitances. */
    for (int e = 0; e < n_nets; ++e) {
        int drv = net_ptr[e];
        double xd = x[pin_cell[drv]] + pin_dx[drv];
        double yd = y[pin_cell[drv]] + pin_dy[drv];
        double load = 0.0;
        tnet[drv] = 0.0;
        for (int s = drv + 1; s < net_ptr[e + 1]; ++s) {
            double xs = x[pin_cell[s]] + pin_dx[s];
            double ys = y[pin_cell[s]] + pin_dy[s];
            double L = fabs(xs - xd) + fabs(ys - yd);
            double R = r * L;
            double Cw = c * L;
            tnet[s] = R * (Cw / 2.0 + pin_cap[s]);
            load += Cw + pin_cap[s];
        }
        cload[e] = load;
        dnet[e] = d0 + cell_rdrv[pin_cell[drv]] * load;
    }

    /* In-degree of every pin in the timing graph. */
    int32_t *indeg = (int32_t *)calloc((size_t)(n_pins > 0 ? n_pins : 1), sizeof(int32_t));
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_pins > 0 ? n_pins : 1));
    if (!indeg || !order) { free(indeg); free(order); nl_free(&nl); return OR_ERR_OOM; }
    for (int p = 0; p < n_pins; ++p) {
        int cell = pin_cell[p];
        if (!is_driver(&nl, p)) {
            indeg[p] = 1;                         /* its net arc */
        } else if (cell_type[cell] == COMB) {
            int k = 0;                            /* one arc per input pin */
            for (int q = nl.cp_ptr[cell]; q < nl.cp_ptr[cell + 1]; ++q)
                if (!is_driver(&nl, nl.cp[q])) ++k;
            indeg[p] = k;
        } else {
            indeg[p] = 0;                         /* startpoint */
        }
    }
    /* Kahn's algorithm: a topological order of the pins. */
    int head = 0, tail = 0;
    for (int p = 0; p < n_pins; ++p)
        if (indeg[p] == 0) order[tail++] = p;
    while (head < tail) {
        int v = order[head++];
        if (is_driver(&nl, v)) {
            int e = nl.pin_net[v];
            for (int s = net_ptr[e] + 1; s < net_ptr[e + 1]; ++s)
                if (--indeg[s] == 0) order[tail++] = s;
        } else if (cell_type[pin_cell[v]] == COMB) {
            int o = comb_output(&nl, pin_cell[v]);
            if (o >= 0 && --indeg[o] == 0) order[tail++] = o;
        }
    }
    if (tail != n_pins) { free(indeg); free(order); nl_free(&nl); return OR_ERR_CYCLE; }

    /* Arr forward in topological order: max over in-arcs, lowest pin on ties. */
    for (int k = 0; k < n_pins; ++k) {
        int v = order[k];
        int cell = pin_cell[v];
        pred[v] = -1;
        if (!is_driver(&nl, v)) {
            int u = net_ptr[nl.pin_net[v]];
            arr[v] = arr[u] + tnet[v];
            pred[v] = u;
        } else if (cell_type[cell] == COMB) {
            double d = dnet[nl.pin_net[v]];
            double best = -INFINITY;
            int bu = -1;
            for (int q = nl.cp_ptr[cell]; q < nl.cp_ptr[cell + 1]; ++q) {
                int u = nl.cp[q];
                if (is_driver(&nl, u)) continue;
                double a = arr[u] + d;
                if (a > best || (a == best && u < bu)) { best = a; bu = u; }
            }
            arr[v] = best;
            pred[v] = bu;
        } else {
            arr[v] = dnet[nl.pin_net[v]];         /* launch at t = 0 plus d */
        }
    }
    /* Req backward in reverse topological order: min over out-arcs. */
    for (int k = n_pins - 1; k >= 0; --k) {
        int v = order[k];
        int cell = pin_cell[v];
        if (is_endpoint(&nl, v)) {
            req[v] = T;
        } else if (is_driver(&nl, v)) {
            int e = nl.pin_net[v];
            double m = INFINITY;
            for (int s = net_ptr[e] + 1; s < net_ptr[e + 1]; ++s) {
                double q = req[s] - tnet[s];
                if (q < m) m = q;
            }
            req[v] = m;
        } else {                                  /* input of a combinational cell */
            int o = comb_output(&nl, cell);
            req[v] = req[o] - dnet[nl.pin_net[o]];
        }
    }
    /* Eq. (2) slack; Eqs. (3)-(4) over the violated endpoints. */
    double w = 0.0, t = 0.0;
    for (int p = 0; p < n_pins; ++p) {
        slack[p] = req[p] - arr[p];
        if (is_endpoint(&nl, p) && slack[p] < 0.0) {
            if (slack[p] < w) w = slack[p];
            t += slack[p];
        }
    }
    *wns = w;
    *tns = t;
    free(indeg); free(order); nl_free(&nl);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* report_timing_endpoint(n, k)  (Section III-B)                             */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t pin;     /* the pin this partial path has reached (going backwards) */
    int32_t parent;  /* state one pin closer to the endpoint, -1 at the endpoint */
    int32_t depth;   /* number of pins from the endpoint to here, inclusive    */
    double S;        /* delay of the suffix from this pin to the endpoint      */
} state_t;

typedef struct {
    state_t *st; int n, cap;
    int32_t *heap; int hn, hcap;
    const double *arr;
    int32_t *bufa, *bufb; int bufcap;
} search_t;

static void seq_of(const search_t *s, int idx, int32_t *buf) {
    int d = s->st[idx].depth;
    for (int k = d - 1; k >= 0; --k) { buf[k] = s->st[idx].pin; idx = s->st[idx].parent; }
}

/* 1 if state a comes before state b: larger exact bound (= lower slack)
 * first; on a tie, the pin sequence from the endpoint compared
 * lexicographically, smaller first. */
static int before(search_t *s, int a, int b) {
    double fa = s->arr[s->st[a].pin] + s->st[a].S;
    double fb = s->arr[s->st[b].pin] + s->st[b].S;
    if (fa != fb) return fa > fb;
    seq_of(s, a, s->bufa);
    seq_of(s, b, s->bufb);
    int da = s->st[a].depth, db = s->st[b].depth;
    int m = da < db ? da : db;
    for (int k = 0; k < m; ++k)
        if (s->bufa[k] != s->bufb[k]) return s->bufa[k] < s->bufb[k];
    return da < db;
}

static int push_state(search_t *s, int pin, int parent, double S) {
    if (s->n == s->cap) {
        int nc = s->cap ? 2 * s->cap : 1024;
        state_t *ns = (state_t *)realloc(s->st, sizeof(state_t) * (size_t)nc);
        if (!ns) return OR_ERR_OOM;
        s->st = ns; s->cap = nc;
    }
    int idx = s->n++;
    s->st[idx].pin = pin;
    s->st[idx].parent = parent;
    s->st[idx].depth = parent < 0 ? 1 : s->st[parent].depth + 1;
    s->st[idx].S = S;
    if (s->st[idx].depth > s->bufcap) {
        int nc = 2 * s->st[idx].depth;
        int32_t *a = (int32_t *)realloc(s->bufa, sizeof(int32_t) * (size_t)nc);
        if (!a) return OR_ERR_OOM;
        s->bufa = a;
        int32_t *b = (int32_t *)realloc(s->bufb, sizeof(int32_t) * (size_t)nc);
        if (!b) return OR_ERR_OOM;
        s->bufb = b;
        s->bufcap = nc;
    }
    if (s->hn == s->hcap) {
        int nc = s->hcap ? 2 * s->hcap : 1024;
        int32_t *nh = (int32_t *)realloc(s->heap, sizeof(int32_t) * (size_t)nc);
        if (!nh) return OR_ERR_OOM;
        s->heap = nh; s->hcap = nc;
    }
    int i = s->hn++;
    s->heap[i] = idx;
    while (i > 0) {                               /* sift up */
        int p = (i - 1) / 2;
        if (!before(s, s->heap[i], s->heap[p])) break;
        int t = s->heap[i]; s->heap[i] = s->heap[p]; s->heap[p] = t;
        i = p;
    }
    return OR_OK;
}

static int pop_state(search_t *s) {
    int top = s->heap[0];
    s->heap[0] = s->heap[--s->hn];
    int i = 0;
    for (;;) {                                    /* sift down */
        int l = 2 * i + 1, r = l + 1, m = i;
        if (l < s->hn && before(s, s->heap[l], s->heap[m])) m = l;
        if (r < s->hn && before(s, s->heap[r], s->heap[m])) m = r;
        if (m == i) break;
        int t = s->heap[i]; s->heap[i] = s->heap[m]; s->heap[m] = t;
        i = m;
    }
    return top;
}

typedef struct {
    int64_t n_paths, n_pins_total;
    int32_t n_viol;
    int32_t *viol;        /* violating endpoints, sorted by (slack, pin) */
    int32_t *ep;          /* per path: its endpoint                     */
    int32_t *rank;        /* per path: 0-based rank within its endpoint */
    double *slack;        /* per path: T - path delay                   */
    int64_t *pin_ptr;     /* per path: offsets into pins (n_paths + 1)  */
    int32_t *pins;        /* path pins, startpoint first, endpoint last */
} or_paths_t;

static const double *g_sort_slack;
static int cmp_ep(const void *a, const void *b) {
    int32_t pa = *(const int32_t *)a, pb = *(const int32_t *)b;
    double sa = g_sort_slack[pa], sb = g_sort_slack[pb];
    if (sa < sb) return -1;
    if (sa > sb) return 1;
    return (pa > pb) - (pa < pb);
}

/*
 * For each of the n most critical failing endpoints (all when n < 0) return
 * its K lowest-slack start->end paths (fewer if it has fewer paths; with
 * keep_nonneg == 0 only paths of negative slack are kept).
 *
 * The search runs backwards from the endpoint.  A state is a partial path
 * from some pin v to the endpoint with suffix delay S; Arr(v) + S is the
 * delay of its best completion, an exact bound because Arr(v) is the largest
 * delay of any path from a startpoint to v.  States are expanded best first,
 * so complete paths leave the queue in order of increasing slack.
 */
/*
 * ep_list / n_list: when n_list >= 0, search exactly these endpoints (in the
 * given order) instead of the n most critical failing ones.
 */
int or_topk(int n_cells, int n_pins, int n_nets, const int32_t *pin_cell, const int32_t *net_ptr,
            const int32_t *cell_type, const double *tnet, const double *dnet, const double *arr,
            double T, int n_endpoints, int K, int keep_nonneg, const int32_t *ep_list, int n_list,
            or_paths_t *out) {
    memset(out, 0, sizeof(*out));
    nl_t nl;
    int st = nl_init(&nl, n_cells, n_pins, n_nets, pin_cell, net_ptr, cell_type);
    if (st) { nl_free(&nl); return st; }

    /* violating endpoints, most critical first */
    int nv = 0;
    int32_t *viol = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_pins > 0 ? n_pins : 1));
    double *eps = (double *)malloc(sizeof(double) * (size_t)(n_pins > 0 ? n_pins : 1));
    if (!viol || !eps) { free(viol); free(eps); nl_free(&nl); return OR_ERR_OOM; }
    for (int p = 0; p < n_pins; ++p) {
        eps[p] = T - arr[p];
        if (is_endpoint(&nl, p) && eps[p] < 0.0) viol[nv++] = p;
    }
    g_sort_slack = eps;
    qsort(viol, (size_t)nv, sizeof(int32_t), cmp_ep);
    int n_use = (n_endpoints < 0 || n_endpoints > nv) ? nv : n_endpoints;

    int64_t pcap = 1024, pincap = 16384;
    out->ep = (int32_t *)malloc(sizeof(int32_t) * (size_t)pcap);
    out->rank = (int32_t *)malloc(sizeof(int32_t) * (size_t)pcap);
    out->slack = (double *)malloc(sizeof(double) * (size_t)pcap);
    out->pin_ptr = (int64_t *)malloc(sizeof(int64_t) * (size_t)(pcap + 1));
    out->pins = (int32_t *)malloc(sizeof(int32_t) * (size_t)pincap);
    if (!out->ep || !out->rank || !out->slack || !out->pin_ptr || !out->pins) goto oom;
    out->pin_ptr[0] = 0;

    search_t s;
    memset(&s, 0, sizeof(s));
    s.arr = arr;
    if (n_list >= 0) n_use = n_list;
    for (int iv = 0; iv < n_use; ++iv) {
        int e = n_list >= 0 ? ep_list[iv] : viol[iv];
        s.n = 0; s.hn = 0;
        if (push_state(&s, e, -1, 0.0)) goto oom_s;
        int found = 0;
        while (s.hn > 0 && found < K) {
            int cur = pop_state(&s);
            int v = s.st[cur].pin;
            double S = s.st[cur].S;
            double path_slack = T - (arr[v] + S);
            if (!keep_nonneg && path_slack >= 0.0) break;
            if (is_startpoint(&nl, v)) {
                /* a complete path: record it, startpoint first */
                int d = s.st[cur].depth;
                if (out->n_paths + 1 >= pcap) {
                    pcap *= 2;
                    out->ep = (int32_t *)realloc(out->ep, sizeof(int32_t) * (size_t)pcap);
                    out->rank = (int32_t *)realloc(out->rank, sizeof(int32_t) * (size_t)pcap);
                    out->slack = (double *)realloc(out->slack, sizeof(double) * (size_t)pcap);
                    out->pin_ptr = (int64_t *)realloc(out->pin_ptr, sizeof(int64_t) * (size_t)(pcap + 1));
                    if (!out->ep || !out->rank || !out->slack || !out->pin_ptr) goto oom_s;
                }
                while (out->n_pins_total + d > pincap) {
                    pincap *= 2;
                    out->pins = (int32_t *)realloc(out->pins, sizeof(int32_t) * (size_t)pincap);
                    if (!out->pins) goto oom_s;
                }
                int idx = cur;
                for (int k = 0; k < d; ++k) {         /* state chain runs start -> endpoint */
                    out->pins[out->n_pins_total + k] = s.st[idx].pin;
                    idx = s.st[idx].parent;
                }
                out->ep[out->n_paths] = e;
                out->rank[out->n_paths] = found;
                out->slack[out->n_paths] = path_slack;
                out->n_pins_total += d;
                out->n_paths += 1;
                out->pin_ptr[out->n_paths] = out->n_pins_total;
                ++found;
                continue;
            }
            if (!is_driver(&nl, v)) {                 /* sink: its net arc */
                int u = net_ptr[nl.pin_net[v]];
                if (push_state(&s, u, cur, S + tnet[v])) goto oom_s;
            } else {                                  /* combinational output: cell arcs */
                int cell = pin_cell[v];
                double d = dnet[nl.pin_net[v]];
                for (int q = nl.cp_ptr[cell]; q < nl.cp_ptr[cell + 1]; ++q) {
                    int u = nl.cp[q];
                    if (is_driver(&nl, u)) continue;
                    if (push_state(&s, u, cur, S + d)) goto oom_s;
                }
            }
        }
    }
    free(s.st); free(s.heap); free(s.bufa); free(s.bufb);
    out->n_viol = nv;
    out->viol = viol;
    free(eps);
    nl_free(&nl);
    return OR_OK;
oom_s:
    free(s.st); free(s.heap); free(s.bufa); free(s.bufb);
oom:
    free(viol); free(eps); nl_free(&nl);
    return OR_ERR_OOM;
}

void or_free_paths(or_paths_t *p) {
    free(p->viol); free(p->ep); free(p->rank); free(p->slack); free(p->pin_ptr); free(p->pins);
    memset(p, 0, sizeof(*p));
}

/* ------------------------------------------------------------------------ */
/* Pin-pair set and weights, Eq. (w_ij)  (Section III-D)                     */
/* ------------------------------------------------------------------------ */

static const double *g_path_slack;
static int cmp_path(const void *a, const void *b) {
    int64_t pa = *(const int64_t *)a, pb = *(const int64_t *)b;
    double sa = g_path_slack[pa], sb = g_path_slack[pb];
    if (sa < sb) return -1;
    if (sa > sb) return 1;
    return (pa > pb) - (pa < pb);
}

/*
 * Traverse the paths worst first.  Every net arc (driver -> sink) on a path
 * is a pin pair, identified by its sink pin (a sink has one driver).  A pair
 * not yet in P enters P with weight w0; a pair already in P gains
 * w1 * slack / WNS, slack being the (negative) slack of the path.
 */
int or_update_pairs(int n_pins, const uint8_t *pin_dir, int64_t n_paths, const double *slack,
                    const int64_t *pin_ptr, const int32_t *pins, double wns, double w0, double w1,
                    uint8_t *in_p, double *w) {
    (void)n_pins;
    if (n_paths == 0 || wns == 0.0) return OR_OK;
    int64_t *ord = (int64_t *)malloc(sizeof(int64_t) * (size_t)n_paths);
    if (!ord) return OR_ERR_OOM;
    for (int64_t k = 0; k < n_paths; ++k) ord[k] = k;
    g_path_slack = slack;
    qsort(ord, (size_t)n_paths, sizeof(int64_t), cmp_path);
    for (int64_t k = 0; k < n_paths; ++k) {
        int64_t q = ord[k];
        for (int64_t j = pin_ptr[q] + 1; j < pin_ptr[q + 1]; ++j) {
            int a = pins[j - 1], b = pins[j];
            if (!(pin_dir[a] == 1 && pin_dir[b] == 0)) continue;   /* cell arc */
            if (!in_p[b]) {
                in_p[b] = 1;
                w[b] = w0;
            } else {
                w[b] += w1 * (slack[q] / wns);
            }
        }
    }
    free(ord);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Pin-to-pin attraction loss (Eq. (9) and PP of Section III-D)             */
/* ------------------------------------------------------------------------ */

/*
 * PP = beta * sum over pairs (drv, s) in P of w_s * Q(drv, s), with
 * Q(i, j) = (x_i - x_j)^2 + (y_i - y_j)^2 on pin coordinates
 * (cell position plus pin offset).  Gradients with respect to cell x / y are
 * added into gx / gy (zeroed first); fixed cells get zero when drop_fixed.
 */
/* Pin-pair distance term of the loss, kind 0: the quadratic Q(i,j) of
 * Eq. (9).  Kinds 1 and 2 are the two alternatives of the ablation
 * (Section IV), which the paper names but does not write out: kind 1 the
 * pair's HPWL |dx| + |dy|, kind 2 its linear Euclidean distance
 * sqrt(dx^2 + dy^2).  Their gradients: sign(dx), sign(dy) (0 at 0) for
 * HPWL; dx / d, dy / d (0 when the pins coincide) for the distance. */
double or_loss_kind(int n_cells, int n_pins, int n_nets, const int32_t *pin_cell,
                    const int32_t *net_ptr, const double *pin_dx, const double *pin_dy,
                    const uint8_t *cell_fixed, const double *x, const double *y, const uint8_t *in_p,
                    const double *w, double beta, int drop_fixed, int kind, double *gx, double *gy) {
    double pp = 0.0;
    for (int c = 0; c < n_cells; ++c) { gx[c] = 0.0; gy[c] = 0.0; }
    (void)n_pins;
    for (int e = 0; e < n_nets; ++e) {
        int drv = net_ptr[e];
        int cd = pin_cell[drv];
        double xd = x[cd] + pin_dx[drv], yd = y[cd] + pin_dy[drv];
        for (int s = drv + 1; s < net_ptr[e + 1]; ++s) {
            if (!in_p[s]) continue;
            int cs = pin_cell[s];
            double xs = x[cs] + pin_dx[s], ys = y[cs] + pin_dy[s];
            double ddx = xs - xd, ddy = ys - yd;
            double term, gxs, gys;
            if (kind == 1) {
                term = fabs(ddx) + fabs(ddy);
                gxs = beta * w[s] * (double)((ddx > 0.0) - (ddx < 0.0));
                gys = beta * w[s] * (double)((ddy > 0.0) - (ddy < 0.0));
            } else if (kind == 2) {
                term = sqrt(ddx * ddx + ddy * ddy);
                gxs = term > 0.0 ? beta * w[s] * ddx / term : 0.0;
                gys = term > 0.0 ? beta * w[s] * ddy / term : 0.0;
            } else {
                term = ddx * ddx + ddy * ddy;
                gxs = 2.0 * beta * w[s] * ddx;
                gys = 2.0 * beta * w[s] * ddy;
            }
            pp += w[s] * term;
            gx[cs] += gxs; gy[cs] += gys;
            gx[cd] -= gxs; gy[cd] -= gys;
        }
    }
    if (drop_fixed)
        for (int c = 0; c < n_cells; ++c)
            if (cell_fixed[c]) { gx[c] = 0.0; gy[c] = 0.0; }
    return beta * pp;
}

double or_loss(int n_cells, int n_pins, int n_nets, const int32_t *pin_cell,
               const int32_t *net_ptr, const double *pin_dx, const double *pin_dy,
               const uint8_t *cell_fixed, const double *x, const double *y, const uint8_t *in_p,
               const double *w, double beta, int drop_fixed, double *gx, double *gy) {
    return or_loss_kind(n_cells, n_pins, n_nets, pin_cell, net_ptr, pin_dx, pin_dy, cell_fixed, x, y,
                        in_p, w, beta, drop_fixed, 0, gx, gy);
}

/* ------------------------------------------------------------------------ */
/* Net weighting from pin slacks (the baseline of Section II-C and of the   */
/* "w/o Path Extraction" ablation, Section IV)                              */
/* ------------------------------------------------------------------------ */

/*
 * The net-weighting scheme the paper compares against (DREAMPlace 4.0's):
 * the placement objective weights each net's wirelength by w_e (Section
 * II-C), a net's weight follows the worst pin slack within the net (the
 * three-pin-net example of Section III-A), and the weights are updated with
 * momentum (Section IV).  The paper gives no constants or formula, so this
 * is a stated reading:
 *   s_e     worst slack over the pins of net e (slack[] from or_sta);
 *   c_e     criticality min(1, max(0, -s_e) / |WNS|), 0 when WNS = 0;
 *   w_e  <- alpha * w_e + (1 - alpha) * (1 + gamma * c_e).
 * w is updated in place; returns the number of nets with s_e < 0.
 */
int or_net_weights(int n_nets, const int32_t *net_ptr, const double *slack, double wns, double alpha,
                   double gamma, double *w) {
    int n_crit = 0;
    for (int e = 0; e < n_nets; ++e) {
        double s = slack[net_ptr[e]];
        for (int p = net_ptr[e] + 1; p < net_ptr[e + 1]; ++p)
            if (slack[p] < s) s = slack[p];
        double c = 0.0;
        if (s < 0.0) {
            ++n_crit;
            if (wns < 0.0) {
                c = -s / -wns;
                if (c > 1.0) c = 1.0;
            }
        }
        w[e] = alpha * w[e] + (1.0 - alpha) * (1.0 + gamma * c);
    }
    return n_crit;
}
