"""attraction_loss_fwd_noalloc against attraction_loss_fwd, through the C ABI.

Callers that cannot allocate device memory (a device-memory budget fixed in
advance, an allocator that owns all device memory, no allocation allowed
after start-up) cannot build a tdp_graph, because sta_build allocates.  The
no-allocation entry point takes every array from the caller and keeps its
partial sums in a static device array of the library.  This file is named so
that pytest collects it last: a run that stops at the first failure has then
already run every other test.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import netgen

pytestmark = pytest.mark.gpu


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def test_noalloc_loss_matches_graph_loss_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import oracle
    from paper_2503_11674_b300 import TimingGraph, _abi
    from paper_2503_11674_b300.build import build

    build()
    lib = _abi.load()
    nl = netgen.generate("diff", 2)
    G = TimingGraph(nl, "fp32")
    rng = np.random.default_rng(11)
    sinks = np.nonzero(nl.pin_dir == 0)[0]
    pins = np.sort(rng.choice(sinks, len(sinks) // 2, replace=False)).astype(np.int32)
    w = rng.uniform(5.0, 20.0, len(pins)).astype(np.float32)
    G.attraction_set_pairs(pins, w.astype(np.float64))
    w_pin = np.zeros(nl.n_pins, np.float32)
    w_pin[pins] = w
    in_p = np.zeros(nl.n_pins, np.uint8)
    in_p[pins] = 1

    dev = torch.device("cuda", torch.cuda.current_device())

    def dv(a, dt):
        return torch.tensor(np.ascontiguousarray(a), dtype=dt, device=dev)

    net_ptr, pin_cell = dv(nl.net_ptr, torch.int32), dv(nl.pin_cell, torch.int32)
    dx, dy, wd = dv(nl.pin_dx, torch.float32), dv(nl.pin_dy, torch.float32), dv(w_pin, torch.float32)
    stream = C.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    beta = 2.5e-5

    def noalloc(n_nets, x, y, out):
        return lib.attraction_loss_fwd_noalloc(n_nets, _ptr(net_ptr), _ptr(pin_cell), _ptr(dx), _ptr(dy),
                                               _ptr(wd), _ptr(x), _ptr(y), beta, _ptr(out), stream)

    for k in range(2):  # two calls in a row, on two placements
        xh = (nl.x + rng.normal(0.0, 5.0, nl.n_cells)).astype(np.float32)
        yh = (nl.y + rng.normal(0.0, 5.0, nl.n_cells)).astype(np.float32)
        x, y = dv(xh, torch.float32), dv(yh, torch.float32)
        ref = G.attraction_loss_fwd(x, y, beta).item()
        # the FP64 oracle on the same (FP32-rounded) positions and weights
        pp, _, _ = oracle.loss(nl, in_p, w_pin.astype(np.float64), beta, xh.astype(np.float64),
                               yh.astype(np.float64))
        out = torch.full((), float("nan"), dtype=torch.float64, device=dev)
        torch.cuda.synchronize(dev)
        free_before = torch.cuda.mem_get_info(dev)[0]
        st = noalloc(nl.n_nets, x, y, out)
        assert st == _abi.TDP_OK, lib.tdp_last_error()
        torch.cuda.synchronize(dev)
        if k == 1:  # the first call may load the library's device code
            assert torch.cuda.mem_get_info(dev)[0] == free_before
        assert out.item() == pytest.approx(ref, rel=1e-6)
        assert out.item() == pytest.approx(pp, rel=1e-6)
        # the same inputs again: the fixed-order reduction gives the same bits
        again = torch.full((), float("nan"), dtype=torch.float64, device=dev)
        assert noalloc(nl.n_nets, x, y, again) == _abi.TDP_OK
        torch.cuda.synchronize(dev)
        assert again.item() == out.item()
    # no nets: the loss is zero
    zero = torch.full((), float("nan"), dtype=torch.float64, device=dev)
    assert noalloc(0, x, y, zero) == _abi.TDP_OK
    torch.cuda.synchronize(dev)
    assert zero.item() == 0.0
    # more nets than the static scratch holds: rejected before any work
    st = noalloc(4_194_305, x, y, out)
    assert st == _abi.TDP_ERR_INVALID
    assert b"static scratch" in lib.tdp_last_error()
