"""Failure paths, made on the host (no device fault is ever made): an injected
device-allocation failure inside hvxVerifyGraph and hvxCreateImage, and a
server request whose launch fails on the host.  The library reports the
failure, keeps the context usable, and every other result stays exact."""
import numpy as np
import pytest

import oracle as O
from paper_2008_11476_gb300 import graphs as PG
from paper_2008_11476_gb300 import hvx as H
from paper_2008_11476_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture
def ctx():
    c = H.hvxCreateContext()
    yield c
    H.hvxTestInjectFault(H.HVX_FAULT_NONE)
    H.hvxReleaseContext(c)


def test_allocation_failure_in_verify_and_create_image(ctx):
    w, h = 640, 360
    img = synth.rects_noise(w, h, seed=71)
    inp = PG.upload(ctx, img, H.HVX_DF_U8)
    ph, mk = PG.empty(ctx, w, h, H.HVX_DF_U8), PG.empty(ctx, w, h, H.HVX_DF_U8)
    # the unfused graph materialises its intermediates at verify time: the
    # first of those allocations fails
    g = PG.edge_graph(ctx, inp, ph, mk, fusion=False, verify=False)
    H.hvxTestInjectFault(H.HVX_FAULT_DEVICE_ALLOC, 1)
    with pytest.raises(H.HvxError) as e:
        H.hvxVerifyGraph(g)
    assert e.value.status == H.HVX_ERROR_NO_MEMORY
    with pytest.raises(H.HvxError) as e:  # not verified: nothing runs
        H.hvxProcessGraph(g)
    assert e.value.status == H.HVX_ERROR_NOT_VERIFIED
    # the fault fired once: the same graph verifies and runs, exactly
    H.hvxVerifyGraph(g)
    H.hvxProcessGraph(g)
    rp, rm = O.edge_graph(img)
    np.testing.assert_array_equal(PG.download(ph), rp)
    np.testing.assert_array_equal(PG.download(mk), rm)
    # an image allocation that fails leaves the context working
    H.hvxTestInjectFault(H.HVX_FAULT_DEVICE_ALLOC, 2)
    PG.empty(ctx, 64, 64, H.HVX_DF_U8)
    with pytest.raises(H.HvxError) as e:
        PG.empty(ctx, 64, 64, H.HVX_DF_U8)
    assert e.value.status == H.HVX_ERROR_NO_MEMORY
    o = PG.empty(ctx, w, h, H.HVX_DF_U8)
    g2 = PG.gaussian_graph(ctx, inp, o)
    H.hvxProcessGraph(g2)
    np.testing.assert_array_equal(PG.download(o), O.gaussian3x3(img).data)


def test_server_request_failing_on_the_host(ctx):
    """Five requests arrive together; the third dispatch fails on the host.
    That request alone reports the failure; the four others complete with
    the results their graphs give alone."""
    jobs = []
    for i in range(5):
        w, h = [(640, 480), (1920, 1080), (333, 97)][i % 3]
        img = synth.rects_noise(w, h, 130 + i)
        inp = PG.upload(ctx, img, H.HVX_DF_U8)
        ph, mk = PG.empty(ctx, w, h, H.HVX_DF_U8), PG.empty(ctx, w, h, H.HVX_DF_U8)
        jobs.append((img, PG.edge_graph(ctx, inp, ph, mk), ph, mk))
    srv = H.hvxCreateServer(ctx, 1 << 30, 8, 4)
    try:
        H.hvxTestInjectFault(H.HVX_FAULT_LAUNCH, 3)
        tickets = H.hvxServerSubmitMany(srv, [j[1] for j in jobs])
        res = [H.hvxServerWait(srv, t, 10000)[0] for t in tickets]
        assert res == [H.HVX_SUCCESS, H.HVX_SUCCESS, H.HVX_ERROR_DEVICE, H.HVX_SUCCESS,
                       H.HVX_SUCCESS]
        st = H.hvxServerStats(srv)
        assert st["completed"] == 4 and st["failed"] == 1
        for k, (img, g, ph, mk) in enumerate(jobs):
            if k == 2:
                continue
            rp, rm = O.edge_graph(img)
            np.testing.assert_array_equal(PG.download(ph), rp)
            np.testing.assert_array_equal(PG.download(mk), rm)
        # the failed request's graph is served normally afterwards
        assert H.hvxServerWait(srv, H.hvxServerSubmit(srv, jobs[2][1]), 10000)[0] == H.HVX_SUCCESS
        rp, rm = O.edge_graph(jobs[2][0])
        np.testing.assert_array_equal(PG.download(jobs[2][2]), rp)
        np.testing.assert_array_equal(PG.download(jobs[2][3]), rm)
    finally:
        H.hvxReleaseServer(srv)
