"""Host-side failure paths through the C ABI, with the failures made on the
host (no GPU is faulted, trapped or stalled):

* out of memory: tdp_debug_fail_alloc makes the n-th next device allocation
  fail without calling CUDA.  sta_build must return TDP_ERR_OOM and free what
  it had allocated, for every allocation it makes; a temporary allocation
  failing inside sta_get_paths, attraction_get_pairs or report_timing must
  return TDP_ERR_OOM and leave the graph usable, with the same results after.
* a level sweep's grid-wide wait that gave up: tdp_debug_set_sync_status
  writes the sticky status word a real timeout sets.  The next
  host-synchronising sta_propagate must return TDP_ERR_TIMEOUT, the results
  must count as invalid (extraction then returns TDP_ERR_STATE), and the next
  propagation must succeed with the same WNS / TNS.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import netgen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2503_11674_b300 import TimingGraph, _abi
    from paper_2503_11674_b300.build import build
    build()
    lib = _abi.load()
    nl = netgen.generate("tiny", 1)
    T = oracle.clock_period(nl, 0.9)
    yield dict(lib=lib, abi=_abi, TG=TimingGraph, nl=nl, T=T)
    lib.tdp_debug_fail_alloc(0)


def _pending(lib):
    n = C.c_int64()
    assert lib.tdp_debug_pending_alloc_failure(C.byref(n)) == 0
    return n.value


def _pos(nl, dev="cuda"):
    return (torch.tensor(nl.x, dtype=torch.float32, device=dev),
            torch.tensor(nl.y, dtype=torch.float32, device=dev))


def test_sta_build_out_of_memory_at_every_allocation(env):
    lib, abi, TG, nl = env["lib"], env["abi"], env["TG"], env["nl"]
    G = TG(nl, "fp32")  # loads the device code; the context's own memory settles
    G.close()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    k = 1
    failed = 0
    while True:
        assert lib.tdp_debug_fail_alloc(k) == abi.TDP_OK
        try:
            G = TG(nl, "fp32")
        except abi.TdpError as e:
            assert e.status == abi.TDP_ERR_OOM, str(e)
            assert _pending(lib) == 0
            failed += 1
            k += 1
            continue
        # fewer allocations than k: the build succeeded with the failure pending
        assert _pending(lib) > 0
        lib.tdp_debug_fail_alloc(0)
        G.close()
        break
    assert failed >= 10, failed
    torch.cuda.synchronize()
    # nothing leaked by the failed builds (device memory is handed out in
    # 2 MiB pages; a leak per failed build would exceed this)
    assert torch.cuda.mem_get_info()[0] >= free0 - (4 << 20)


def test_temporary_allocations_fail_cleanly(env):
    lib, abi, TG, nl, T = env["lib"], env["abi"], env["TG"], env["nl"], env["T"]
    G = TG(nl, "fp32")
    x, y = _pos(nl)
    G.sta_propagate(x, y, T)
    G.extract_critical_paths(-1, 4, False)
    ref = {k: v.cpu().numpy() for k, v in G.sta_get_paths().items()}
    n_pairs = G.attraction_update_pairs(10.0, 0.2)
    pins_ref, w_ref = (t.cpu().numpy() for t in G.attraction_get_pairs())
    # sta_get_paths: sort, scans and materialisation temporaries
    for k in (1, 2, 3, 4, 5, 6, 7, 8):
        G.extract_critical_paths(-1, 4, False)
        lib.tdp_debug_fail_alloc(k)
        try:
            got = {kk: v.cpu().numpy() for kk, v in G.sta_get_paths().items()}
        except abi.TdpError as e:
            assert e.status == abi.TDP_ERR_OOM, str(e)
            lib.tdp_debug_fail_alloc(0)
            continue
        lib.tdp_debug_fail_alloc(0)
        for kk in ref:
            np.testing.assert_array_equal(got[kk], ref[kk])
    got = {kk: v.cpu().numpy() for kk, v in G.sta_get_paths().items()}
    for kk in ref:
        np.testing.assert_array_equal(got[kk], ref[kk])
    # attraction_get_pairs: flag and offset temporaries
    lib.tdp_debug_fail_alloc(1)
    with pytest.raises(abi.TdpError) as ei:
        G.attraction_get_pairs()
    assert ei.value.status == abi.TDP_ERR_OOM
    lib.tdp_debug_fail_alloc(0)
    pins, w = (t.cpu().numpy() for t in G.attraction_get_pairs())
    assert len(pins) == n_pairs
    np.testing.assert_array_equal(pins, pins_ref)
    np.testing.assert_array_equal(w, w_ref)
    # report_timing: its node store and rounds
    n_ref = G.report_timing(20)
    rep_ref = {kk: v.cpu().numpy() for kk, v in G.sta_get_paths().items()}
    oom = 0
    for k in range(1, 12):
        lib.tdp_debug_fail_alloc(k)
        try:
            G.report_timing(20)
        except abi.TdpError as e:
            assert e.status == abi.TDP_ERR_OOM, str(e)
            oom += 1
        lib.tdp_debug_fail_alloc(0)
    assert oom >= 3
    assert G.report_timing(20) == n_ref
    rep = {kk: v.cpu().numpy() for kk, v in G.sta_get_paths().items()}
    for kk in ("ep", "slack", "pin_ptr", "pins"):
        np.testing.assert_array_equal(rep[kk], rep_ref[kk])
    G.close()


def test_grid_wait_timeout_status_maps_to_timeout(env):
    lib, abi, TG, nl, T = env["lib"], env["abi"], env["TG"], env["nl"], env["T"]
    G = TG(nl, "fp32")
    x, y = _pos(nl)
    wns, tns = G.sta_propagate(x, y, T)
    assert lib.tdp_debug_set_sync_status(G.handle, 1) == abi.TDP_OK
    with pytest.raises(abi.TdpError) as ei:
        G.sta_propagate(x, y, T)
    assert ei.value.status == abi.TDP_ERR_TIMEOUT
    assert "gave up" in str(ei.value)
    # the results of the call that timed out are invalid: no extraction
    with pytest.raises(abi.TdpError) as ei:
        G.extract_critical_paths(-1, 4, False)
    assert ei.value.status == abi.TDP_ERR_STATE
    # the word was cleared: the next propagation succeeds, with the same bits
    assert G.sta_propagate(x, y, T) == (wns, tns)
    assert G.extract_critical_paths(-1, 4, False) > 0
    # the status is also checked by an extraction that synchronises
    assert lib.tdp_debug_set_sync_status(G.handle, 1) == abi.TDP_OK
    with pytest.raises(abi.TdpError) as ei:
        G.extract_critical_paths(-1, 4, False)
    assert ei.value.status == abi.TDP_ERR_TIMEOUT
    assert G.sta_propagate(x, y, T) == (wns, tns)
    G.close()
