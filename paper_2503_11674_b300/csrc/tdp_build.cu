// sta_build / sta_destroy: validate the netlist, levelize the combinational
// cells (the timing graph of Section II-B is a DAG once flip-flops cut it),
// and lay the level-ordered CSR arrays out in device memory.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <cstring>
#include <numeric>

#include "tdp_internal.cuh"

namespace tdp {

static thread_local char g_err[1024] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

template <typename T>
static tdp_status upload(tdp_graph *g, T **dst, const std::vector<T> &src) {
    TDP_TRY(dalloc(g, dst, src.size()));
    if (!src.empty())
        TDP_CUDA(cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
    return TDP_OK;
}

template <typename R>
static tdp_status build_state(tdp_graph *g, const tdp_netlist_desc *d) {
    State<R> &s = state<R>(g);
    Topo &t = g->topo;
    using A = typename Acc<R>::T;
    std::vector<R> v(d->pin_dx, d->pin_dx + t.n_pins);
    TDP_TRY(upload(g, &s.pin_dx, v));
    v.assign(d->pin_dy, d->pin_dy + t.n_pins);
    TDP_TRY(upload(g, &s.pin_dy, v));
    v.assign(d->pin_cap, d->pin_cap + t.n_pins);
    TDP_TRY(upload(g, &s.pin_cap, v));
    v.assign(d->cell_rdrv, d->cell_rdrv + t.n_cells);
    TDP_TRY(upload(g, &s.cell_rdrv, v));
    TDP_TRY(dalloc(g, &s.tnet, t.n_pins));
    TDP_TRY(dalloc(g, &s.cload, t.n_nets));
    TDP_TRY(dalloc(g, &s.dnet, t.n_nets));
    TDP_TRY(dalloc(g, &s.arr, t.n_pins));
    TDP_TRY(dalloc(g, &s.req, t.n_pins));
    TDP_TRY(dalloc(g, &s.slack, t.n_pins));
    TDP_TRY(dalloc(g, &s.T, 1));
    TDP_TRY(dalloc(g, &s.wns_tns, 2));
    TDP_TRY(dalloc(g, &s.red_part, 2 * ((size_t)t.n_ep / kRedChunk + 1)));
    TDP_TRY(dalloc(g, &s.red_count, 1));
    TDP_CUDA(cudaMemset(s.red_count, 0, sizeof(unsigned)));
    TDP_TRY(dalloc(g, &s.gsync, 4));
    TDP_CUDA(cudaMemset(s.gsync, 0, 4 * sizeof(unsigned)));
    TDP_CUDA(cudaMemset(s.tnet, 0, sizeof(R) * t.n_pins));
    // static per-net path data of startpoints: no worst input, chain length 1
    std::vector<int32_t> pred(t.n_nets, -1), plen(t.n_nets, 1);
    {
        std::vector<int2> pr(t.n_nets, make_int2(-1, -1));
        TDP_TRY(upload(g, &s.pred, pr));
    }
    TDP_TRY(upload(g, &s.plen, plen));
    // extraction
    TDP_TRY(dalloc(g, &s.sort_a, 2 * (size_t)std::max(t.n_ep, 1)));
    TDP_TRY(dalloc(g, &s.sort_b, 2 * (size_t)std::max(t.n_ep, 1)));
    TDP_TRY(dalloc(g, &s.nviol, 1));
    TDP_TRY(dalloc(g, &s.viol, std::max(t.n_ep, 1)));
    TDP_TRY(dalloc(g, &s.ep_flag, (size_t)t.n_ep + 32));
    TDP_CUDA(cudaMemset(s.ep_flag, 0, (size_t)t.n_ep + 32));
    TDP_TRY(dalloc(g, &s.bcnt, t.n_nets));
    TDP_CUDA(cudaMemset(s.bcnt, 0, sizeof(int32_t) * t.n_nets));
    TDP_TRY(dalloc(g, &s.p_count, std::max(t.n_ep, 1)));
    TDP_TRY(dalloc(g, &s.n_paths, 1));
    // pin pairs
    TDP_TRY(dalloc(g, &s.sumq, t.n_pins));
    TDP_TRY(dalloc(g, &s.maxq, t.n_pins));
    TDP_TRY(dalloc(g, &s.in_p, t.n_pins));
    TDP_TRY(dalloc(g, &s.w, t.n_pins));
    TDP_TRY(dalloc(g, &s.n_pairs, 1));
    TDP_CUDA(cudaMemset(s.sumq, 0, sizeof(long long) * t.n_pins));
    std::vector<long long> mq(t.n_pins, INT64_MIN);
    TDP_CUDA(cudaMemcpy(s.maxq, mq.data(), sizeof(long long) * t.n_pins, cudaMemcpyHostToDevice));
    TDP_CUDA(cudaMemset(s.in_p, 0, t.n_pins));
    TDP_CUDA(cudaMemset(s.w, 0, sizeof(R) * t.n_pins));
    TDP_CUDA(cudaMemset(s.n_pairs, 0, sizeof(long long)));
    // backward sweep: required time keys of the nets
    TDP_TRY(dalloc(g, &s.reqkey, t.n_nets));
    // loss
    TDP_TRY(dalloc(g, &s.net_pf, (size_t)t.n_nets + 32));
    TDP_TRY(dalloc(g, &s.cell_pf, (size_t)t.n_cells + 32));
    TDP_TRY(dalloc(g, &s.ppins, std::max(t.n_pins, 1)));
    TDP_TRY(dalloc(g, &s.pcells, t.n_cells));
    {
        const size_t ns = (size_t)std::max(t.n_pins - t.n_nets, 1);
        TDP_TRY(dalloc(g, &s.pr_a, ns));
        TDP_TRY(dalloc(g, &s.pr_o, 4 * ns));
        TDP_TRY(dalloc(g, &s.pr_w, ns));
        TDP_TRY(dalloc(g, &s.pr_n, ns));
        TDP_TRY(dalloc(g, &s.pr_big, (size_t)std::max(t.n_big, 1)));
        TDP_TRY(dalloc(g, &s.pr_nbig, 1));
        TDP_CUDA(cudaMemset(s.pr_nbig, 0, sizeof(int32_t)));
    }
    TDP_TRY(dalloc(g, &s.pcnt, 2));
    TDP_TRY(dalloc(g, &s.cmp_tiles, compact_tile_cap(t)));
    TDP_CUDA(cudaMemset(s.cmp_tiles, 0, sizeof(unsigned long long) * compact_tile_cap(t)));
    TDP_TRY(dalloc(g, &s.cmp_ctr, 2));
    TDP_CUDA(cudaMemset(s.cmp_ctr, 0, 2 * sizeof(unsigned)));
    TDP_CUDA(cudaMemset(s.net_pf, 0, (size_t)t.n_nets + 32));
    TDP_CUDA(cudaMemset(s.cell_pf, 0, (size_t)t.n_cells + 32));
    TDP_CUDA(cudaMemset(s.pcnt, 0, 2 * sizeof(int32_t)));
    TDP_TRY(dalloc(g, &s.gslot, 2 * (size_t)t.n_pins));
    TDP_CUDA(cudaMemset(s.gslot, 0, 2 * sizeof(R) * (size_t)t.n_pins));
    TDP_TRY(dalloc(g, &s.loss_part, 1024));
    TDP_TRY(dalloc(g, &s.loss_count, 1));
    TDP_CUDA(cudaMemset(s.loss_count, 0, sizeof(unsigned)));
    (void)sizeof(A);
    return TDP_OK;
}

static bool finite_nonneg(float v) { return std::isfinite(v) && v >= 0.0f; }

static tdp_status build_topology(tdp_graph *g, const tdp_netlist_desc *d) {
    Topo &t = g->topo;
    const int nc = d->n_cells, np = d->n_pins, nn = d->n_nets;
    if (nc <= 0 || np <= 0 || nn <= 0 || np > kBwPinMask) {
        set_error("sta_build: n_cells, n_pins and n_nets must be positive, n_pins below 2^28");
        return TDP_ERR_INVALID;
    }
    if (!d->pin_cell || !d->net_ptr || !d->pin_dir || !d->cell_type || !d->pin_dx ||
        !d->pin_dy || !d->pin_cap || !d->cell_rdrv || !d->cell_fixed) {
        set_error("sta_build: a netlist array pointer is NULL");
        return TDP_ERR_INVALID;
    }
    if (!(std::isfinite(d->r_per_um) && d->r_per_um >= 0 && std::isfinite(d->c_per_um) &&
          d->c_per_um >= 0 && std::isfinite(d->d0_ps) && d->d0_ps >= 0)) {
        set_error("sta_build: r_per_um, c_per_um and d0_ps must be finite and >= 0");
        return TDP_ERR_INVALID;
    }
    if (d->net_ptr[0] != 0 || d->net_ptr[nn] != np) {
        set_error("sta_build: net_ptr must start at 0 and end at n_pins");
        return TDP_ERR_INVALID;
    }
    std::vector<int32_t> pin_net(np);
    int n_big = 0;
    for (int e = 0; e < nn; ++e) {
        int a = d->net_ptr[e], b = d->net_ptr[e + 1];
        if (b - a < 2 || a < 0 || b > np) {
            set_error("sta_build: net %d has %d pins (needs a driver and at least one sink)", e,
                      b - a);
            return TDP_ERR_INVALID;
        }
        if (b - a - 1 > kBigFanout) ++n_big;
        for (int p = a; p < b; ++p) {
            pin_net[p] = e;
            if (d->pin_dir[p] != (p == a ? 1 : 0)) {
                set_error("sta_build: pin %d of net %d: pin_dir must be 1 for the first pin and 0 "
                          "for the others", p, e);
                return TDP_ERR_INVALID;
            }
        }
    }
    for (int c = 0; c < nc; ++c) {
        int ty = d->cell_type[c];
        if (ty < TDP_CELL_COMB || ty > TDP_CELL_PO) {
            set_error("sta_build: cell %d has unknown type %d", c, ty);
            return TDP_ERR_INVALID;
        }
        if (!finite_nonneg(d->cell_rdrv[c])) {
            set_error("sta_build: cell %d has a non-finite or negative drive resistance", c);
            return TDP_ERR_INVALID;
        }
    }
    std::vector<int32_t> n_in(nc, 0), n_out(nc, 0), out_pin(nc, -1);
    for (int p = 0; p < np; ++p) {
        int c = d->pin_cell[p];
        if (c < 0 || c >= nc) {
            set_error("sta_build: pin %d refers to cell %d out of range", p, c);
            return TDP_ERR_INVALID;
        }
        if (!finite_nonneg(d->pin_cap[p]) || !std::isfinite(d->pin_dx[p]) ||
            !std::isfinite(d->pin_dy[p])) {
            set_error("sta_build: pin %d has a non-finite offset or capacitance", p);
            return TDP_ERR_INVALID;
        }
        if (d->pin_dir[p]) {
            n_out[c]++;
            out_pin[c] = p;
        } else {
            n_in[c]++;
        }
    }
    int n_comb = 0;
    for (int c = 0; c < nc; ++c) {
        int ty = d->cell_type[c];
        bool ok = true;
        if (ty == TDP_CELL_COMB) {
            ok = n_in[c] >= 1 && n_in[c] <= kMaxFanin && n_out[c] == 1;
            ++n_comb;
        } else if (ty == TDP_CELL_FF) {
            ok = n_in[c] <= 1 && n_out[c] <= 1;
        } else if (ty == TDP_CELL_PI) {
            ok = n_in[c] == 0 && n_out[c] == 1;
        } else {
            ok = n_in[c] == 1 && n_out[c] == 0;
        }
        if (!ok) {
            set_error("sta_build: cell %d (type %d) has %d inputs and %d outputs", c, ty, n_in[c],
                      n_out[c]);
            return TDP_ERR_INVALID;
        }
    }
    // cell -> pins CSR, ascending pin index
    std::vector<int32_t> cp_ptr(nc + 1, 0), cp(np), slot(np);
    for (int p = 0; p < np; ++p) cp_ptr[d->pin_cell[p] + 1]++;
    for (int c = 0; c < nc; ++c) cp_ptr[c + 1] += cp_ptr[c];
    {
        std::vector<int32_t> fill(cp_ptr.begin(), cp_ptr.end() - 1);
        for (int p = 0; p < np; ++p) {
            int k = fill[d->pin_cell[p]]++;
            cp[k] = p;
            slot[p] = k;
        }
    }
    // levelize combinational cells (Kahn); flip-flops and primary inputs are level 0
    std::vector<int32_t> level(nc, 0), deps(nc, 0);
    for (int c = 0; c < nc; ++c) {
        if (d->cell_type[c] != TDP_CELL_COMB) continue;
        level[c] = 1;
        for (int k = cp_ptr[c]; k < cp_ptr[c + 1]; ++k) {
            int p = cp[k];
            if (d->pin_dir[p]) continue;
            int dc = d->pin_cell[d->net_ptr[pin_net[p]]];
            if (d->cell_type[dc] == TDP_CELL_COMB) deps[c]++;
        }
    }
    std::vector<int32_t> queue;
    queue.reserve(n_comb);
    for (int c = 0; c < nc; ++c)
        if (d->cell_type[c] == TDP_CELL_COMB && deps[c] == 0) queue.push_back(c);
    for (size_t h = 0; h < queue.size(); ++h) {
        int c = queue[h];
        int e = pin_net[out_pin[c]];
        for (int s = d->net_ptr[e] + 1; s < d->net_ptr[e + 1]; ++s) {
            int c2 = d->pin_cell[s];
            if (d->cell_type[c2] != TDP_CELL_COMB) continue;
            level[c2] = std::max(level[c2], level[c] + 1);
            if (--deps[c2] == 0) queue.push_back(c2);
        }
    }
    if ((int)queue.size() != n_comb) {
        set_error("sta_build: combinational loop (%d of %d combinational cells levelized)",
                  (int)queue.size(), n_comb);
        return TDP_ERR_CYCLE;
    }
    int D = 0;
    for (int c = 0; c < nc; ++c)
        if (d->cell_type[c] == TDP_CELL_COMB) D = std::max(D, level[c]);

    // combinational cells by (level, id)
    std::vector<int32_t> lvl_ptr(D + 1, 0);
    for (int c = 0; c < nc; ++c)
        if (d->cell_type[c] == TDP_CELL_COMB) lvl_ptr[level[c]]++;
    for (int l = 1; l <= D; ++l) lvl_ptr[l] += lvl_ptr[l - 1];
    // lvl_ptr[l] = number of cells with level <= l; cells of level l: [lvl_ptr[l-1], lvl_ptr[l])
    std::vector<int32_t> lv_cell(n_comb);
    {
        std::vector<int32_t> fill(D + 1, 0);
        for (int l = 1; l <= D; ++l) fill[l] = lvl_ptr[l - 1];
        for (int c = 0; c < nc; ++c)
            if (d->cell_type[c] == TDP_CELL_COMB) lv_cell[fill[level[c]]++] = c;
    }
    std::vector<int32_t> lv_out(n_comb), lv_onet(n_comb), lv_in_ptr(n_comb + 1, 0);
    std::vector<int32_t> lv_in_pin, lv_in_drv, lv_in_net;
    std::vector<uint8_t> lv_in_flags;
    for (int k = 0; k < n_comb; ++k) {
        int c = lv_cell[k];
        lv_out[k] = out_pin[c];
        lv_onet[k] = pin_net[out_pin[c]];
        for (int q = cp_ptr[c]; q < cp_ptr[c + 1]; ++q) {
            int p = cp[q];
            if (d->pin_dir[p]) continue;
            lv_in_pin.push_back(p);
            lv_in_drv.push_back(d->net_ptr[pin_net[p]]);
            lv_in_net.push_back(pin_net[p]);
            const int dc = d->pin_cell[d->net_ptr[pin_net[p]]];
            lv_in_flags.push_back((d->cell_type[dc] == TDP_CELL_COMB ? kInComb : 0) |
                                  (level[dc] == level[c] - 1 ? kInPrev : 0));
        }
        lv_in_ptr[k + 1] = (int32_t)lv_in_pin.size();
    }
    // per-pin kinds and sink links
    std::vector<uint8_t> kind(np);
    std::vector<int32_t> sink_out(np, -1), sink_onet(np, -1), ep;
    for (int p = 0; p < np; ++p) {
        int c = d->pin_cell[p];
        int ty = d->cell_type[c];
        if (d->pin_dir[p]) {
            kind[p] = (ty == TDP_CELL_COMB) ? PK_COMB_OUT : PK_START;
        } else if (ty == TDP_CELL_COMB) {
            kind[p] = PK_COMB_IN;
            sink_out[p] = out_pin[c];
            sink_onet[p] = pin_net[out_pin[c]];
        } else {
            kind[p] = PK_ENDPOINT;
            ep.push_back(p);
        }
    }
    // nets grouped by driver level; small nets first within a level
    std::vector<int32_t> net_level(nn);
    for (int e = 0; e < nn; ++e) net_level[e] = level[d->pin_cell[d->net_ptr[e]]];
    std::vector<int32_t> bl_ptr(D + 2, 0), bl_small(D + 1, 0), bl_net(nn), big;
    for (int e = 0; e < nn; ++e) {
        bl_ptr[net_level[e] + 1]++;
        if (d->net_ptr[e + 1] - d->net_ptr[e] - 1 <= kBigFanout) bl_small[net_level[e]]++;
        else big.push_back(e);
    }
    for (int l = 0; l <= D; ++l) bl_ptr[l + 1] += bl_ptr[l];
    {
        std::vector<int32_t> fs(D + 1), fb(D + 1);
        for (int l = 0; l <= D; ++l) {
            fs[l] = bl_ptr[l];
            fb[l] = bl_ptr[l] + bl_small[l];
        }
        for (int e = 0; e < nn; ++e) {
            int l = net_level[e];
            bool small = d->net_ptr[e + 1] - d->net_ptr[e] - 1 <= kBigFanout;
            bl_net[small ? fs[l]++ : fb[l]++] = e;
        }
    }
    // backward warp tasks per level, deepest level first: tasks of small nets
    // (at most kBwSmallFanout sinks), a net on an aligned group of 1, 2 or 4
    // lanes (kBwPerLane sinks a lane: sinks j and j + G of a net of G lanes
    // on its lane j), the groups of 4 first, then of 2, then single lanes,
    // packed 32 lanes a task; then pieces of kBwPiece sinks of the larger nets
    // (sinks l and l + 32 of the piece on lane l).  Per task and lane: the
    // net's driver pin (kBwSplit set when the net has several pieces, kBwG2 /
    // kBwG4 for groups of 2 / 4 lanes; -1: none) and the net; per task and
    // lane, kBwPerLane sink slots (pin, kind | kKindPrev, net driven by the
    // sink's cell; pin -1: none).
    std::vector<int2> bw_drv;
    std::vector<int4> bw_slot;
    const int4 no_slot = make_int4(-1, 0, 0, 0);
    auto slot_of = [&](int p) {
        int fl = kind[p];
        if (kind[p] == PK_COMB_IN && level[d->pin_cell[p]] == net_level[pin_net[p]] + 1) fl |= kKindPrev;
        return make_int4(p, fl, sink_onet[p], 0);
    };
    std::vector<int4> bw_lv(D + 1);  // (first task, small-net tasks, piece tasks, 0)
    int n_tasks = 0;
    for (int l = D; l >= 0; --l) {
        const int first = n_tasks;
        std::vector<int32_t> small, large;
        for (int q = bl_ptr[l]; q < bl_ptr[l + 1]; ++q) {
            const int e = bl_net[q];
            (d->net_ptr[e + 1] - d->net_ptr[e] - 1 <= kBwSmallFanout ? small : large).push_back(e);
        }
        int lane = 0;  // next lane of the current task
        for (int G : {4, 2, 1}) {
            for (int e : small) {
                const int a = d->net_ptr[e], b = d->net_ptr[e + 1];
                const int ns = b - a - 1;
                if ((ns > 2 * kBwPerLane ? 4 : ns > kBwPerLane ? 2 : 1) != G) continue;
                if (lane == 0) ++n_tasks;
                for (int ln = 0; ln < G; ++ln) {
                    bw_drv.push_back(make_int2(a | (G == 4 ? kBwG4 : G == 2 ? kBwG2 : 0), e));
                    for (int j = 0; j < kBwPerLane; ++j) {
                        const int p = a + 1 + ln + j * G;
                        bw_slot.push_back(p < b ? slot_of(p) : no_slot);
                    }
                }
                lane = (lane + G) & 31;  // groups stay aligned: larger groups come first
            }
        }
        for (; lane != 0; lane = (lane + 1) & 31) {  // the last task's unused lanes
            bw_drv.push_back(make_int2(-1, -1));
            for (int j = 0; j < kBwPerLane; ++j) bw_slot.push_back(no_slot);
        }
        const int n_small_tasks = n_tasks - first;
        for (int e : large) {
            const int a = d->net_ptr[e], b = d->net_ptr[e + 1];
            const int parts = (b - a - 1 + kBwPiece - 1) / kBwPiece;
            for (int j = 0; j < parts; ++j, ++n_tasks) {
                const int p0 = a + 1 + j * kBwPiece, p1 = std::min(b, p0 + kBwPiece);
                for (int ln = 0; ln < 32; ++ln) {
                    bw_drv.push_back(make_int2(a | (parts > 1 ? kBwSplit : 0), e));
                    for (int jj = 0; jj < kBwPerLane; ++jj) {
                        const int p = p0 + ln + jj * 32;
                        bw_slot.push_back(p < p1 ? slot_of(p) : no_slot);
                    }
                }
            }
        }
        bw_lv[l] = make_int4(first, n_small_tasks, n_tasks - first - n_small_tasks, 0);
    }
    t.n_bw_tasks = n_tasks;
    TDP_TRY(upload(g, &t.bw_drv, bw_drv));
    TDP_TRY(upload(g, &t.bw_slot, bw_slot));
    TDP_TRY(upload(g, &t.bw_lv, bw_lv));
    std::vector<int32_t> s_lo(D + 1), s_n(D + 1), b_lo(D + 1), b_n(D + 1);
    for (int l = 0; l <= D; ++l) {
        s_lo[l] = bw_lv[l].x;
        s_n[l] = bw_lv[l].y;
        b_lo[l] = bw_lv[l].x + bw_lv[l].y;
        b_n[l] = bw_lv[l].z;
    }
    t.n_cells = nc;
    t.n_pins = np;
    t.n_nets = nn;
    t.n_comb = n_comb;
    t.n_in = (int32_t)lv_in_pin.size();
    t.n_ep = (int32_t)ep.size();
    t.depth = D;
    t.n_big = (int32_t)big.size();
    g->lv.lvl_ptr = lvl_ptr;
    g->lv.bw_s_lo = s_lo;
    g->lv.bw_s_n = s_n;
    g->lv.bw_b_lo = b_lo;
    g->lv.bw_b_n = b_n;
    TDP_TRY(upload(g, &t.lvl_ptr, lvl_ptr));
    std::vector<int32_t> pc(d->pin_cell, d->pin_cell + np), nptr(d->net_ptr, d->net_ptr + nn + 1);
    std::vector<uint8_t> fixed(d->cell_fixed, d->cell_fixed + nc);
    TDP_TRY(upload(g, &t.pin_cell, pc));
    TDP_TRY(upload(g, &t.pin_net, pin_net));
    TDP_TRY(upload(g, &t.net_ptr, nptr));
    TDP_TRY(upload(g, &t.pin_kind, kind));
    TDP_TRY(upload(g, &t.sink_out, sink_out));
    TDP_TRY(upload(g, &t.sink_onet, sink_onet));
    TDP_TRY(upload(g, &t.net_level, net_level));
    TDP_TRY(upload(g, &t.big_nets, big));
    TDP_TRY(upload(g, &t.lv_out, lv_out));
    TDP_TRY(upload(g, &t.lv_onet, lv_onet));
    TDP_TRY(upload(g, &t.lv_in_ptr, lv_in_ptr));
    TDP_TRY(upload(g, &t.lv_in_pin, lv_in_pin));
    TDP_TRY(upload(g, &t.lv_in_drv, lv_in_drv));
    TDP_TRY(upload(g, &t.lv_in_net, lv_in_net));
    TDP_TRY(upload(g, &t.lv_in_flags, lv_in_flags));
    {
        std::vector<int4> rec(n_comb), slot((size_t)n_comb * kPre, make_int4(-1, -1, -1, 0));
        for (int k = 0; k < n_comb; ++k) {
            const int a = lv_in_ptr[k], nin = lv_in_ptr[k + 1] - a;
            rec[k] = make_int4(lv_onet[k], lv_out[k], nin, a);
            for (int u = 0; u < nin && nin <= kPre; ++u)
                slot[(size_t)k * kPre + u] = make_int4(lv_in_pin[a + u], lv_in_net[a + u], lv_in_drv[a + u],
                                                       lv_in_flags[a + u]);
        }
        TDP_TRY(upload(g, &t.lv_rec, rec));
        TDP_TRY(upload(g, &t.lv_slot, slot));
    }
    TDP_TRY(upload(g, &t.ep, ep));
    {
        std::vector<int2> ep_pd(ep.size());
        for (size_t i = 0; i < ep.size(); ++i) ep_pd[i] = make_int2(ep[i], d->net_ptr[pin_net[ep[i]]]);
        TDP_TRY(upload(g, &t.ep_pd, ep_pd));
    }
    TDP_TRY(upload(g, &t.cp_ptr, cp_ptr));
    TDP_TRY(upload(g, &t.cp, cp));
    TDP_TRY(upload(g, &t.slot_of_pin, slot));
    TDP_TRY(upload(g, &t.cell_fixed, fixed));
    return TDP_OK;
}

}  // namespace tdp

namespace tdp {

const char *const kKernelNames[KID_COUNT] = {"net_rc",    "fwd_sweep",   "bwd_sweep", "viol_sort",
                                              "topk",      "pair_walk",   "pair_finish", "pp_fwd",
                                              "pp_bwd_net", "pp_bwd_cell", "rt_expand", "ep_wns",
                                              "inc_moved", "fwd_inc",     "net_weights", "pp_fwd_bwd"};

static cudaEvent_t prof_event(tdp_graph *g) {
    if (!g->prof_free.empty()) {
        cudaEvent_t e = g->prof_free.back();
        g->prof_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

LaunchScope::LaunchScope(tdp_graph *g_, KernelId id, int n_kernels, cudaStream_t st_)
    : g(g_), on(g_->prof_id == id), st(st_ ? st_ : g_->stream) {
    g->n_launch += n_kernels;
    if (on) {
        a = prof_event(g);
        if (a) cudaEventRecord(a, st);
    }
}

LaunchScope::~LaunchScope() {
    if (!on || !a) return;
    cudaEvent_t b = prof_event(g);
    if (!b) return;
    cudaEventRecord(b, st);
    g->prof_pending.emplace_back(a, b);
}

void join_side(tdp_graph *g) {
    if (!g->bwd_pending) return;
    cudaStreamWaitEvent(g->stream, g->ev_bwd, 0);
    g->bwd_pending = false;
}

}  // namespace tdp

namespace tdp {

tdp_status check_sync_status(tdp_graph *g) {
    join_side(g);  // the status word covers the backward sweep too
    unsigned *w = g->prec == TDP_FP32 ? g->s32.gsync : g->s64.gsync;
    unsigned h = 0;
    TDP_CUDA(cudaMemcpyAsync(&h, w + 1, sizeof(h), cudaMemcpyDeviceToHost, g->stream));
    TDP_CUDA(cudaStreamSynchronize(g->stream));
    if (h == 0) return TDP_OK;
    TDP_CUDA(cudaMemsetAsync(w + 1, 0, sizeof(unsigned), g->stream));
    g->propagated = false;
    g->extracted = false;
    g->inc_valid = false;
    set_error("a level sweep's grid-wide wait gave up after %.1f s; timing results are not valid",
              kSyncTimeoutNs * 1e-9);
    return TDP_ERR_TIMEOUT;
}

}  // namespace tdp

using namespace tdp;

extern "C" const char *tdp_last_error(void) { return g_err; }

extern "C" tdp_status tdp_get_launch_count(tdp_graph *g, int64_t *n_out) {
    if (!g || !n_out) {
        set_error("tdp_get_launch_count: NULL argument");
        return TDP_ERR_INVALID;
    }
    *n_out = g->n_launch;
    return TDP_OK;
}

extern "C" tdp_status tdp_profile_kernel(tdp_graph *g, const char *name) {
    if (!g) {
        set_error("tdp_profile_kernel: NULL graph");
        return TDP_ERR_INVALID;
    }
    int id = -1;
    if (name && name[0]) {
        for (int k = 0; k < KID_COUNT; ++k)
            if (!strcmp(name, kKernelNames[k])) id = k;
        if (id < 0) {
            set_error("tdp_profile_kernel: unknown kernel name '%s'", name);
            return TDP_ERR_INVALID;
        }
    }
    g->prof_id = id;
    return TDP_OK;
}

extern "C" tdp_status tdp_profile_read(tdp_graph *g, int64_t *launches_out, double *total_ms_out) {
    if (!g) {
        set_error("tdp_profile_read: NULL graph");
        return TDP_ERR_INVALID;
    }
    TDP_CUDA(cudaStreamSynchronize(g->stream));
    if (g->side) TDP_CUDA(cudaStreamSynchronize(g->side));
    double total = 0.0;
    for (auto &pr : g->prof_pending) {
        float ms = 0.0f;
        TDP_CUDA(cudaEventElapsedTime(&ms, pr.first, pr.second));
        total += ms;
        g->prof_free.push_back(pr.first);
        g->prof_free.push_back(pr.second);
    }
    if (launches_out) *launches_out = (int64_t)g->prof_pending.size();
    if (total_ms_out) *total_ms_out = total;
    g->prof_pending.clear();
    return TDP_OK;
}

extern "C" void sta_destroy(tdp_graph *g) {
    if (!g) return;
    if (g->side) cudaStreamSynchronize(g->side);
    if (g->fwd_graph) cudaGraphExecDestroy(g->fwd_graph);
    if (g->bwd_graph) cudaGraphExecDestroy(g->bwd_graph);
    for (auto &pr : g->prof_pending) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    for (cudaEvent_t e : g->prof_free) cudaEventDestroy(e);
    rt_free(g);
    for (void *p : g->allocs) cudaFree(p);
    if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
    if (g->side) cudaStreamDestroy(g->side);
    if (g->ev_bwd_go) cudaEventDestroy(g->ev_bwd_go);
    if (g->ev_bwd) cudaEventDestroy(g->ev_bwd);
    delete g;
}

extern "C" tdp_status sta_build(const tdp_netlist_desc *netlist, tdp_precision precision,
                                void *cuda_stream, tdp_graph **out) {
    if (!out) {
        set_error("sta_build: out is NULL");
        return TDP_ERR_INVALID;
    }
    *out = nullptr;
    if (!netlist) {
        set_error("sta_build: netlist is NULL");
        return TDP_ERR_INVALID;
    }
    if (precision != TDP_FP32 && precision != TDP_FP64) {
        set_error("sta_build: unknown precision %d", (int)precision);
        return TDP_ERR_INVALID;
    }
    tdp_graph *g = new (std::nothrow) tdp_graph();
    if (!g) {
        set_error("sta_build: host allocation failed");
        return TDP_ERR_OOM;
    }
    g->prec = precision;
    g->stream = static_cast<cudaStream_t>(cuda_stream);
    g->r = netlist->r_per_um;
    g->c = netlist->c_per_um;
    g->d0 = netlist->d0_ps;
    tdp_status st = build_topology(g, netlist);
    if (st == TDP_OK) {
        cudaError_t e = cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking);
        // the backward sweep's stream at the highest priority: its blocks are
        // placed before those of the kernels queued beside it
        int prio_lo = 0, prio_hi = 0;
        if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&g->side, cudaStreamNonBlocking, prio_hi);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->ev_bwd_go, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->ev_bwd, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            set_error("sta_build: stream or event creation failed: %s", cudaGetErrorString(e));
            st = TDP_ERR_CUDA;
        }
        // TDP_SERIAL_BWD=1: the backward sweep on the graph's stream, in order
        const char *ser = getenv("TDP_SERIAL_BWD");
        g->overlap_bwd = !(ser && ser[0] == '1');
        const char *share = getenv("TDP_BWD_SHARE");
        if (share) g->bwd_share = std::min(16, std::max(1, atoi(share)));
        const char *bsms = getenv("TDP_BWD_SMS");
        if (bsms) g->bwd_sms = atoi(bsms);
    }
    if (st == TDP_OK)
        st = precision == TDP_FP32 ? build_state<float>(g, netlist) : build_state<double>(g, netlist);
    if (st == TDP_OK) {
        // single-launch level sweeps need cooperative launches; the
        // environment variable TDP_LEVEL_GRAPHS=1 selects the per-level graphs
        int dev = 0, coop = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g->n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        if (e != cudaSuccess) {
            set_error("sta_build: %s", cudaGetErrorString(e));
            st = TDP_ERR_CUDA;
        }
        const char *env = getenv("TDP_LEVEL_GRAPHS");
        g->single_launch = coop != 0 && !(env && env[0] == '1');
    }
    if (st == TDP_OK) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) {
            set_error("sta_build: %s", cudaGetErrorString(e));
            st = TDP_ERR_CUDA;
        }
    }
    if (st != TDP_OK) {
        sta_destroy(g);
        return st;
    }
    *out = g;
    return TDP_OK;
}

// ------------------------------------------------------------ test hooks ---

namespace tdp {
namespace {
std::atomic<int64_t> g_fail_alloc{0};  // n > 0: the n-th next allocation fails
}  // namespace

bool alloc_fail_injected() {
    int64_t c = g_fail_alloc.load();
    while (c > 0) {
        if (g_fail_alloc.compare_exchange_weak(c, c - 1)) return c == 1;
    }
    return false;
}
}  // namespace tdp

extern "C" tdp_status tdp_debug_fail_alloc(int64_t n) {
    if (n < 0) {
        set_error("tdp_debug_fail_alloc: n < 0");
        return TDP_ERR_INVALID;
    }
    g_fail_alloc.store(n);
    return TDP_OK;
}

extern "C" tdp_status tdp_debug_pending_alloc_failure(int64_t *n_out) {
    if (!n_out) {
        set_error("tdp_debug_pending_alloc_failure: n_out is NULL");
        return TDP_ERR_INVALID;
    }
    *n_out = g_fail_alloc.load();
    return TDP_OK;
}

extern "C" tdp_status tdp_debug_set_sync_status(tdp_graph *g, uint32_t status) {
    if (!g) {
        set_error("tdp_debug_set_sync_status: NULL graph");
        return TDP_ERR_INVALID;
    }
    join_side(g);
    unsigned *w = g->prec == TDP_FP32 ? g->s32.gsync : g->s64.gsync;
    const unsigned h = status;
    TDP_CUDA(cudaMemcpyAsync(w + 1, &h, sizeof(h), cudaMemcpyHostToDevice, g->stream));
    TDP_CUDA(cudaStreamSynchronize(g->stream));
    return TDP_OK;
}
