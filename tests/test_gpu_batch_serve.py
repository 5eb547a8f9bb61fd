"""GPU tests of the batched persistent launch and of the serving loop: every
result equals the oracle's and the result of the same graph run alone."""
import numpy as np
import pytest

import oracle as O
from paper_2008_11476_gb300 import graphs as PG
from paper_2008_11476_gb300 import hvx as H
from paper_2008_11476_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = H.hvxCreateContext()
    yield c
    H.hvxReleaseContext(c)


def _edge_set(ctx, sizes, seed):
    items = []
    for i, (w, h) in enumerate(sizes):
        img = synth.rects_noise(w, h, seed + i)
        inp = PG.upload(ctx, img, H.HVX_DF_U8)
        ph = PG.empty(ctx, w, h, H.HVX_DF_U8)
        mk = PG.empty(ctx, w, h, H.HVX_DF_U8)
        g = PG.edge_graph(ctx, inp, ph, mk)
        items.append((img, g, ph, mk))
    return items


def test_batch_uneven_sizes_matches_oracle(ctx):
    sizes = synth.batch_sizes(24, seed=4, wlo=1, whi=700, hlo=1, hhi=400)
    sizes += [(1, 1), (1920, 1080), (321, 2)]
    items = _edge_set(ctx, sizes, 40)
    graphs = [it[1] for it in items]
    for _ in range(2):  # the second call replays the captured CUDA graph
        H.hvxProcessGraphBatch(graphs)
        H.hvxWaitBatch(ctx)
        for img, g, ph, mk in items:
            rp, rm = O.edge_graph(img)
            np.testing.assert_array_equal(PG.download(mk), rm)
            np.testing.assert_array_equal(PG.download(ph), rp)


@pytest.mark.parametrize("rows", [5, 10, 15])
@pytest.mark.parametrize("border", [H.HVX_BORDER_REPLICATE, H.HVX_BORDER_CONSTANT,
                                    H.HVX_BORDER_UNDEFINED])
def test_batch_every_tile_height(monkeypatch, rows, border):
    """The persistent edge kernel with 128 x 8R tiles for each R the tuner can
    choose, on uneven sizes (ragged tiles in both directions) and every
    border: exact against the oracle."""
    monkeypatch.setenv("HVX_BATCH_ROWS", str(rows))
    c = H.hvxCreateContext()
    try:
        sizes = synth.batch_sizes(6, seed=40 + rows, wlo=1, whi=600, hlo=1, hhi=300)
        sizes += [(1, 1), (640, 481), (130, 41)]
        items = []
        for i, (w, h) in enumerate(sizes):
            img = synth.rects_noise(w, h, seed=500 + i)
            inp = PG.upload(c, img, H.HVX_DF_U8)
            ph, mk = PG.empty(c, w, h, H.HVX_DF_U8), PG.empty(c, w, h, H.HVX_DF_U8)
            items.append((img, PG.edge_graph(c, inp, ph, mk, border=border, cval=9), ph, mk))
        graphs = [it[1] for it in items]
        H.hvxProcessGraphBatch(graphs)
        H.hvxWaitBatch(c)
        got_rows, grid = H.hvxQueryBatch(graphs)
        assert got_rows == [rows] * len(items) and grid > 0
        B = {H.HVX_BORDER_REPLICATE: O.BORDER_REPLICATE, H.HVX_BORDER_CONSTANT: O.BORDER_CONSTANT,
             H.HVX_BORDER_UNDEFINED: O.BORDER_UNDEFINED}[border]
        for img, g, ph, mk in items:
            rp, rm = O.edge_graph(img, B, 9)
            np.testing.assert_array_equal(PG.download(mk), rm)
            np.testing.assert_array_equal(PG.download(ph), rp)
    finally:
        H.hvxReleaseContext(c)


def test_batch_shape_tuner_choice_is_exact(ctx):
    """The tuner's own choice (per size class, by timed trials) on a batch with
    all three classes: one R of 5 / 10 / 15 per class, exact results."""
    sizes = [(700, 300), (500, 200), (900, 700), (640, 1000), (1920, 1080), (1500, 1300)]
    items = _edge_set(ctx, sizes, 90)
    graphs = [it[1] for it in items]
    H.hvxProcessGraphBatch(graphs)
    H.hvxWaitBatch(ctx)
    rows, grid = H.hvxQueryBatch(graphs)
    cls = [0 if h < 480 else 1 if h < 1080 else 2 for _, h in sizes]
    for k in set(cls):
        assert len({r for r, c in zip(rows, cls) if c == k}) == 1
    assert set(rows) <= {5, 10, 15} and grid > 0
    for img, g, ph, mk in items:
        rp, rm = O.edge_graph(img)
        np.testing.assert_array_equal(PG.download(mk), rm)
        np.testing.assert_array_equal(PG.download(ph), rp)


def test_batch_gaussian_only(ctx):
    sizes = [(33, 7), (640, 480), (129, 300)]
    outs = []
    graphs = []
    for i, (w, h) in enumerate(sizes):
        img = synth.uniform_u8(w, h, 60 + i)
        o = PG.empty(ctx, w, h, H.HVX_DF_U8)
        graphs.append(PG.gaussian_graph(ctx, PG.upload(ctx, img, H.HVX_DF_U8), o))
        outs.append((img, o))
    H.hvxProcessGraphBatch(graphs)
    H.hvxWaitBatch(ctx)
    for img, o in outs:
        np.testing.assert_array_equal(PG.download(o), O.gaussian3x3(img).data)


@pytest.mark.parametrize("border", [H.HVX_BORDER_REPLICATE, H.HVX_BORDER_CONSTANT,
                                    H.HVX_BORDER_UNDEFINED])
def test_batch_gaussian_every_border(ctx, border):
    # the persistent Gaussian kernel, whose warps fix the border cells of
    # their own rows without a block barrier: edge tiles on all four sides,
    # ragged tiles, images smaller than a tile, every border mode, exact
    sizes = [(1, 1), (7, 3), (128, 120), (129, 121), (300, 250), (1000, 241)]
    B = {H.HVX_BORDER_REPLICATE: O.BORDER_REPLICATE, H.HVX_BORDER_CONSTANT: O.BORDER_CONSTANT,
         H.HVX_BORDER_UNDEFINED: O.BORDER_UNDEFINED}[border]
    outs, graphs = [], []
    for i, (w, h) in enumerate(sizes):
        img = synth.rects_noise(w, h, seed=80 + i)
        o = PG.empty(ctx, w, h, H.HVX_DF_U8)
        graphs.append(PG.gaussian_graph(ctx, PG.upload(ctx, img, H.HVX_DF_U8), o, border=border,
                                        cval=201))
        outs.append((img, o))
    assert PG.kernel_kinds(graphs[0]) == ["gaussian3x3_tma"]
    H.hvxProcessGraphBatch(graphs)
    H.hvxWaitBatch(ctx)
    for img, o in outs:
        ref = O.gaussian3x3(img, B, 201)
        got = PG.download(o)
        x0, y0, x1, y1 = ref.rect
        np.testing.assert_array_equal(got[y0:y1, x0:x1], ref.data[y0:y1, x0:x1])


def test_batch_mixed_kinds_falls_back_to_sequential(ctx):
    img = synth.rects_noise(100, 60, 70)
    inp = PG.upload(ctx, img, H.HVX_DF_U8)
    mk = PG.empty(ctx, 100, 60, H.HVX_DF_U8)
    g1 = PG.harris_graph(ctx, inp, mk)
    g2o = PG.empty(ctx, 100, 60, H.HVX_DF_U8)
    g2 = PG.gaussian_graph(ctx, inp, g2o)
    H.hvxProcessGraphBatch([g1, g2])
    H.hvxWaitBatch(ctx)
    np.testing.assert_array_equal(PG.download(mk), O.harris_graph(img)[0])
    np.testing.assert_array_equal(PG.download(g2o), O.gaussian3x3(img).data)


def test_server_mix_equals_alone(ctx):
    """Requests that arrive together are admitted together (several in flight
    at once, on several streams); each output is the same as when its graph
    runs alone."""
    rng_sizes = [(640, 480), (1920, 1080), (333, 97)]
    jobs = []
    for i in range(9):
        w, h = rng_sizes[i % 3]
        img = synth.rects_noise(w, h, 80 + i)
        inp = PG.upload(ctx, img, H.HVX_DF_U8)
        kind = i % 3
        if kind == 0:
            o = PG.empty(ctx, w, h, H.HVX_DF_U8)
            g = PG.gaussian_graph(ctx, inp, o)
            outs = [o]
        elif kind == 1:
            ph, mk = PG.empty(ctx, w, h, H.HVX_DF_U8), PG.empty(ctx, w, h, H.HVX_DF_U8)
            g = PG.edge_graph(ctx, inp, ph, mk)
            outs = [ph, mk]
        else:
            mk = PG.empty(ctx, w, h, H.HVX_DF_U8)
            g = PG.harris_graph(ctx, inp, mk)
            outs = [mk]
        jobs.append((g, outs))
    alone = []
    for g, outs in jobs:
        H.hvxProcessGraph(g)
        alone.append([PG.download(o) for o in outs])
        for o in outs:  # clear, so the served run must write everything again
            z = np.zeros_like(alone[-1][0])
            H.hvxCopyImage(o, z.ctypes.data, z.strides[0], H.HVX_WRITE)
    srv = H.hvxCreateServer(ctx, 1 << 30, 8, 4)
    tickets = H.hvxServerSubmitMany(srv, [g for g, _ in jobs])
    for t in tickets:
        st, lat = H.hvxServerWait(srv, t, 10000)
        assert st == H.HVX_SUCCESS and lat > 0
    for (g, outs), ref in zip(jobs, alone):
        for o, r in zip(outs, ref):
            np.testing.assert_array_equal(PG.download(o), r)
    stats = H.hvxServerStats(srv)
    assert stats["completed"] == 9 and stats["failed"] == 0
    # the nine arrived together: the dispatcher admits all eight slots' worth
    # in one pass, before any completion is retired
    assert stats["max_in_flight"] == 8
    assert stats["p99_ms"] >= stats["p50_ms"] > 0
    H.hvxReleaseServer(srv)


def test_server_busy_graph_does_not_block_others(ctx):
    """Two requests on one graph and one on another arrive together: the
    second request on the busy graph waits for the first, while the request
    on the other graph is admitted at once (three in flight would need the
    same graph twice).  Every result equals the oracle."""
    w, h = 1920, 1080
    imgs = [synth.rects_noise(w, h, 120 + i) for i in range(2)]
    gs, outs = [], []
    for img in imgs:
        inp = PG.upload(ctx, img, H.HVX_DF_U8)
        ph, mk = PG.empty(ctx, w, h, H.HVX_DF_U8), PG.empty(ctx, w, h, H.HVX_DF_U8)
        gs.append(PG.edge_graph(ctx, inp, ph, mk))
        outs.append((ph, mk))
    srv = H.hvxCreateServer(ctx, 1 << 30, 8, 4)
    tickets = H.hvxServerSubmitMany(srv, [gs[0], gs[0], gs[1]])
    for t in tickets:
        assert H.hvxServerWait(srv, t, 10000)[0] == H.HVX_SUCCESS
    st = H.hvxServerStats(srv)
    assert st["completed"] == 3 and st["max_in_flight"] == 2
    for img, (ph, mk) in zip(imgs, outs):
        rp, rm = O.edge_graph(img)
        np.testing.assert_array_equal(PG.download(ph), rp)
        np.testing.assert_array_equal(PG.download(mk), rm)
    with pytest.raises(H.HvxError):  # all or nothing
        H.hvxServerSubmitMany(srv, [gs[0], None])
    assert H.hvxServerStats(srv)["submitted"] == 3
    H.hvxReleaseServer(srv)


def test_server_budget_admission(ctx):
    """With a budget that holds one request, requests run one at a time and
    all complete; a request larger than the budget is refused."""
    w, h = 512, 256
    jobs = []
    for i in range(4):
        img = synth.rects_noise(w, h, 90 + i)
        inp = PG.upload(ctx, img, H.HVX_DF_U8)
        ph, mk = PG.empty(ctx, w, h, H.HVX_DF_U8), PG.empty(ctx, w, h, H.HVX_DF_U8)
        jobs.append((img, PG.edge_graph(ctx, inp, ph, mk), ph, mk))
    one = 3 * w * h + 1024
    srv = H.hvxCreateServer(ctx, one, 8, 4)
    tickets = [H.hvxServerSubmit(srv, j[1]) for j in jobs]
    for t in tickets:
        assert H.hvxServerWait(srv, t, 10000)[0] == H.HVX_SUCCESS
    st = H.hvxServerStats(srv)
    assert st["max_in_flight"] == 1 and st["peak_bytes_reserved"] <= one
    for img, g, ph, mk in jobs:
        rp, rm = O.edge_graph(img)
        np.testing.assert_array_equal(PG.download(mk), rm)
    H.hvxReleaseServer(srv)
    small = H.hvxCreateServer(ctx, 1000, 4, 1)
    with pytest.raises(H.HvxError) as e:
        H.hvxServerSubmit(small, jobs[0][1])
    assert e.value.status == H.HVX_ERROR_OVER_BUDGET
    H.hvxReleaseServer(small)


def test_image_from_torch_tensor_and_swap(ctx):
    torch = pytest.importorskip("torch")
    w, h = 1000, 300
    pitch = 1024
    a = synth.rects_noise(w, h, 95)
    b = synth.rects_noise(w, h, 96)
    ta = torch.zeros((h, pitch), dtype=torch.uint8, device="cuda")
    tb = torch.zeros((h, pitch), dtype=torch.uint8, device="cuda")
    ta[:, :w] = torch.from_numpy(a).cuda()
    tb[:, :w] = torch.from_numpy(b).cuda()
    to = torch.zeros((h, pitch), dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    inp = H.hvxCreateImageFromHandle(ctx, w, h, H.HVX_DF_U8, ta.data_ptr(), pitch)
    out = H.hvxCreateImageFromHandle(ctx, w, h, H.HVX_DF_U8, to.data_ptr(), pitch)
    g = PG.gaussian_graph(ctx, inp, out)
    H.hvxProcessGraph(g)
    np.testing.assert_array_equal(to[:, :w].cpu().numpy(), O.gaussian3x3(a).data)
    H.hvxSwapImageHandle(inp, tb.data_ptr(), pitch)  # next frame, graph stays verified
    H.hvxProcessGraph(g)
    np.testing.assert_array_equal(to[:, :w].cpu().numpy(), O.gaussian3x3(b).data)


def test_bench_configuration_64_frames_1080p(ctx):
    """The launch configuration bench.py times: 64 frames of 1920x1080 in one
    batched persistent launch; sampled frames (first, middle, last, each with
    its own content) are compared whole with the oracle."""
    F, w, h = 64, 1920, 1080
    distinct = [synth.rects_noise(w, h, seed=2 + i) for i in range(8)]
    graphs, outs = [], []
    for i in range(F):
        inp = PG.upload(ctx, distinct[i % 8], H.HVX_DF_U8)
        ph, mk = PG.empty(ctx, w, h, H.HVX_DF_U8), PG.empty(ctx, w, h, H.HVX_DF_U8)
        graphs.append(PG.edge_graph(ctx, inp, ph, mk))
        outs.append((ph, mk))
    for _ in range(2):
        H.hvxProcessGraphBatch(graphs)
    H.hvxWaitBatch(ctx)
    for i in (0, 5, 31, 63):
        rp, rm = O.edge_graph(distinct[i % 8])
        np.testing.assert_array_equal(PG.download(outs[i][0]), rp)
        np.testing.assert_array_equal(PG.download(outs[i][1]), rm)
    for g in graphs:
        H.hvxReleaseGraph(g)


def test_device_bounded_wait_reports_timeout_and_context_survives(ctx):
    assert H.hvxSelfTestBoundedWait(ctx) == H.HVX_ERROR_TIMEOUT
    # the error word was cleared when it was read, and work still runs
    img = synth.uniform_u8(100, 50, 3)
    inp = PG.upload(ctx, img, H.HVX_DF_U8)
    out = PG.empty(ctx, 100, 50, H.HVX_DF_U8)
    g = PG.gaussian_graph(ctx, inp, out)
    H.hvxProcessGraph(g)
    np.testing.assert_array_equal(PG.download(out), O.gaussian3x3(img).data)


def test_batch_on_host_data(ctx):
    # hvxScheduleGraphBatchHost: host frames in, fused batch, both outputs
    # back, on a stream; pageable numpy memory works too (slower copies)
    from paper_2008_11476_gb300 import hvx as HX
    w, h, n = 320, 240, 5
    frames = [synth.rects_noise(w, h, seed=60 + i) for i in range(n)]
    graphs, items, outs = [], [], []
    for f in frames:
        src = PG.empty(ctx, w, h, HX.HVX_DF_U8)
        ph = PG.empty(ctx, w, h, HX.HVX_DF_U8)
        mk = PG.empty(ctx, w, h, HX.HVX_DF_U8)
        graphs.append(PG.edge_graph(ctx, src, ph, mk))
        hp = np.zeros((h, w), np.uint8)
        hm = np.zeros((h, w), np.uint8)
        outs.append((hp, hm))
        items += [(src, f.ctypes.data, w, True), (ph, hp.ctypes.data, w, False),
                  (mk, hm.ctypes.data, w, False)]
    copies = HX.host_copies(items)
    HX.hvxScheduleGraphBatchHost(graphs, copies)
    HX.hvxWaitBatch(ctx)
    for f, (hp, hm) in zip(frames, outs):
        ref_ph, ref_mk = O.edge_graph(f)
        np.testing.assert_array_equal(hp, ref_ph)
        np.testing.assert_array_equal(hm, ref_mk)
    bad = HX.host_copies([(PG.empty(ctx, w, h, HX.HVX_DF_U8), outs[0][0].ctypes.data, w - 1,
                           True)])
    with pytest.raises(HX.HvxError):  # host pitch below the row size
        HX.hvxScheduleGraphBatchHost(graphs, bad)


@pytest.mark.parametrize("mix", ["harris", "tomasi", "both"])
def test_harris_batch_one_launch(ctx, mix):
    # BORDER_UNDEFINED corner graphs of different sizes in one launch (one
    # rows-per-thread for all of them): the same masks as one launch each.
    # Harris and Shi-Tomasi graphs run different kernels: a batch of both
    # falls back to one launch per graph, with the same results
    sizes = [(1920, 1080), (333, 77), (640, 480), (1, 1), (129, 300), (500, 260)]
    graphs, outs, refs = [], [], []
    for i, (w, h) in enumerate(sizes):
        img = synth.rects_noise(w, h, seed=80 + i)
        src = PG.upload(ctx, img, H.HVX_DF_U8)
        mk = PG.empty(ctx, w, h, H.HVX_DF_U8)
        tomasi = mix == "tomasi" or (mix == "both" and i % 2 == 1)
        g = PG.harris_graph(ctx, src, mk, thr=4.0e4 if tomasi else 1e6, tomasi=tomasi)
        assert PG.kernel_kinds(g) == ["fused_harris_tma"]
        graphs.append(g)
        outs.append(mk)
        refs.append(None if tomasi else O.harris_graph(img)[0])
    singles = []
    for g, mk in zip(graphs, outs):
        H.hvxProcessGraph(g)
        singles.append(PG.download(mk))
    for mk in outs:  # clear the outputs so the batch must write them
        z = np.zeros((H.hvxQueryImage(mk)[1], H.hvxQueryImage(mk)[0]), np.uint8)
        H.hvxCopyImage(mk, z.ctypes.data, z.strides[0], H.HVX_WRITE)
    for want, ref in zip(singles, refs):
        if ref is not None:
            np.testing.assert_array_equal(want, ref)
    if mix != "harris":
        assert singles[-1].any() and not singles[-1].all()
    for _ in range(2):
        H.hvxProcessGraphBatch(graphs)
        H.hvxWaitBatch(ctx)
        for mk, want in zip(outs, singles):
            np.testing.assert_array_equal(PG.download(mk), want)


def test_server_requests_on_host_data(ctx):
    # hvxServerSubmitHost: each request copies its frame in, runs, copies both
    # outputs out; a completed request's results are in host memory
    w, h = 320, 200
    srv = H.hvxCreateServer(ctx, 1 << 30, 4, 2)
    graphs, bufs = [], []
    for i in range(3):
        src = PG.empty(ctx, w, h, H.HVX_DF_U8)
        ph = PG.empty(ctx, w, h, H.HVX_DF_U8)
        mk = PG.empty(ctx, w, h, H.HVX_DF_U8)
        graphs.append((PG.edge_graph(ctx, src, ph, mk), src, ph, mk))
    tickets = []
    for k in range(9):
        g, src, ph, mk = graphs[k % 3]
        f = synth.rects_noise(w, h, seed=200 + k)
        hp = np.zeros((h, w), np.uint8)
        hm = np.zeros((h, w), np.uint8)
        copies = H.host_copies([(src, f.ctypes.data, w, True), (ph, hp.ctypes.data, w, False),
                                (mk, hm.ctypes.data, w, False)])
        bufs.append((f, hp, hm, copies))
        tickets.append(H.hvxServerSubmitHost(srv, g, copies))
        if k % 3 == 2:  # a graph runs one request at a time: wait before reusing it
            for t in tickets[-3:]:
                st, _ = H.hvxServerWait(srv, t)
                assert st == H.HVX_SUCCESS
    for f, hp, hm, _ in bufs:
        rp, rm = O.edge_graph(f)
        np.testing.assert_array_equal(hp, rp)
        np.testing.assert_array_equal(hm, rm)
    H.hvxReleaseServer(srv)


def test_batches_from_two_host_threads(ctx):
    # two threads issue batch calls on one context (shared batch cache) on
    # their own streams; every output stays exact
    import threading
    import torch
    w, h = 256, 144
    sets = []
    for k in range(2):
        graphs, refs, outs = [], [], []
        for i in range(4):
            img = synth.rects_noise(w, h, seed=300 + 10 * k + i)
            src = PG.upload(ctx, img, H.HVX_DF_U8)
            ph, mk = PG.empty(ctx, w, h, H.HVX_DF_U8), PG.empty(ctx, w, h, H.HVX_DF_U8)
            graphs.append(PG.edge_graph(ctx, src, ph, mk))
            refs.append(O.edge_graph(img))
            outs.append((ph, mk))
        sets.append((graphs, refs, outs))
    errors = []

    def work(k):
        try:
            st = torch.cuda.Stream()
            graphs, refs, outs = sets[k]
            for _ in range(20):
                H.hvxProcessGraphBatch(graphs, st.cuda_stream)
            H.hvxWaitBatch(ctx, st.cuda_stream)
            for (rp, rm), (ph, mk) in zip(refs, outs):
                assert np.array_equal(PG.download(ph), rp) and np.array_equal(PG.download(mk), rm)
        except Exception as e:  # reported to the main thread
            errors.append(e)

    ts = [threading.Thread(target=work, args=(k,)) for k in range(2)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not errors, errors


def test_calls_from_a_fresh_host_thread(ctx):
    # a thread that has made no CUDA call yet: the batch call encodes its
    # tensor maps and the generated kernel launches through the driver API,
    # both in that thread
    import threading
    w, h = 300, 170
    img = synth.rects_noise(w, h, seed=404)
    src = PG.upload(ctx, img, H.HVX_DF_U8)
    mk = PG.empty(ctx, w, h, H.HVX_DF_U8)
    gh = PG.harris_graph(ctx, src, mk, thr=4.0e4, tomasi=True)
    out = PG.empty(ctx, w, h, H.HVX_DF_U8)
    gg = H.hvxCreateGraph(ctx)
    m = H.hvxCreateVirtualImage(gg)
    H.hvxSetNodeBorder(H.hvxMedian3x3Node(gg, src, m), H.HVX_BORDER_REPLICATE, 0)
    H.hvxAbsDiffNode(gg, m, src, out)
    H.hvxVerifyGraph(gg)
    assert H.hvxQueryGraph(gg, H.HVX_GRAPH_GENERATED_KERNELS) == 1
    errors = []

    def work():
        try:
            for _ in range(3):
                H.hvxProcessGraphBatch([gh])
                H.hvxWaitBatch(ctx)
                H.hvxProcessGraph(gg)
        except Exception as e:  # reported to the main thread
            errors.append(e)

    t = threading.Thread(target=work)
    t.start()
    t.join()
    assert not errors, errors
    med = O.morph3x3(img, O.MORPH_MEDIAN, O.BORDER_REPLICATE)
    want = O.arith(med, img, np.uint8, O.ARITH_ABSDIFF)
    np.testing.assert_array_equal(PG.download(out), want.data)
    got = PG.download(mk)
    assert got.any() and not got.all()
