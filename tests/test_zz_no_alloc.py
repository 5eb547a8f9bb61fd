"""hvxEdgeBatchNoAlloc: the batched edge graph for callers that cannot allocate
device memory.  Its output must equal hvxProcessGraphBatch's on the same
frames, on two calls in a row (the fixed scratch array is reused and must be
rewritten correctly each time).  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2008_11476_gb300 import graphs as PG
from paper_2008_11476_gb300 import hvx as H
from paper_2008_11476_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("border", [H.HVX_BORDER_REPLICATE, H.HVX_BORDER_UNDEFINED,
                                    H.HVX_BORDER_CONSTANT])
def test_no_alloc_batch_equals_graph_batch_twice(border):
    ctx = H.hvxCreateContext()
    try:
        sizes = synth.batch_sizes(7, seed=11, wlo=1, whi=900, hlo=1, hhi=500)
        sizes += [(1920, 1080), (2, 3)]
        graphs, ref_imgs, frames, outs = [], [], [], []
        for i, (w, h) in enumerate(sizes):
            img = synth.rects_noise(w, h, seed=300 + i)
            inp = PG.upload(ctx, img, H.HVX_DF_U8)
            ph, mk = PG.empty(ctx, w, h, H.HVX_DF_U8), PG.empty(ctx, w, h, H.HVX_DF_U8)
            graphs.append(PG.edge_graph(ctx, inp, ph, mk, border=border, cval=0, thr=100))
            ref_imgs.append((ph, mk))
            ph2, mk2 = PG.empty(ctx, w, h, H.HVX_DF_U8), PG.empty(ctx, w, h, H.HVX_DF_U8)
            ip, ipitch = H.hvxGetImageDevicePtr(inp)
            pp, ppitch = H.hvxGetImageDevicePtr(ph2)
            mp, mpitch = H.hvxGetImageDevicePtr(mk2)
            frames.append(H.hvx_edge_frame(ip, ipitch, pp, ppitch, mp, mpitch, w, h))
            outs.append((ph2, mk2))
        H.hvxProcessGraphBatch(graphs)
        H.hvxWaitBatch(ctx)
        ref = [(PG.download(a), PG.download(b)) for a, b in ref_imgs]
        for call in range(2):
            for a, b in outs:  # stale results must not survive into the check
                z = np.full((H.hvxQueryImage(a)[1], H.hvxQueryImage(a)[0]), 7, np.uint8)
                H.hvxCopyImage(a, z.ctypes.data, z.strides[0], H.HVX_WRITE)
                H.hvxCopyImage(b, z.ctypes.data, z.strides[0], H.HVX_WRITE)
            H.hvxEdgeBatchNoAlloc(frames, border, 100)
            for (a, b), (rp, rm) in zip(outs, ref):
                np.testing.assert_array_equal(PG.download(a), rp, err_msg=f"phase, call {call}")
                np.testing.assert_array_equal(PG.download(b), rm, err_msg=f"mask, call {call}")
    finally:
        H.hvxReleaseContext(ctx)


def test_no_alloc_rejects_too_many_frames_and_bad_frames():
    ctx = H.hvxCreateContext()
    try:
        inp = PG.empty(ctx, 64, 8, H.HVX_DF_U8)
        out = PG.empty(ctx, 64, 8, H.HVX_DF_U8)
        ip, pitch = H.hvxGetImageDevicePtr(inp)
        op, _ = H.hvxGetImageDevicePtr(out)
        f = H.hvx_edge_frame(ip, pitch, op, pitch, None, 0, 64, 8)
        with pytest.raises(H.HvxError) as e:
            H.hvxEdgeBatchNoAlloc([f] * (H.HVX_NOALLOC_MAX_FRAMES + 1), 1, 100)
        assert e.value.status == H.HVX_ERROR_OVER_BUDGET
        bad = H.hvx_edge_frame(ip + 1, pitch, op, pitch, None, 0, 64, 8)
        with pytest.raises(H.HvxError) as e:
            H.hvxEdgeBatchNoAlloc([bad], 1, 100)
        assert e.value.status == H.HVX_ERROR_INVALID_PARAMETERS
    finally:
        H.hvxReleaseContext(ctx)
