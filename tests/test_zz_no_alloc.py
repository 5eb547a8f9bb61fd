"""hvxEdgeBatchNoAlloc: the batched edge graph for callers that cannot allocate
device memory (a process whose device memory belongs to another allocator, a
real-time loop that cannot take cudaMalloc's implicit synchronisation).  Its
output must equal hvxProcessGraphBatch's on the same frames, and the oracle's,
on two calls in a row with different frames, frame counts and borders: the
fixed scratch array is reused, so every table in it must be rewritten
correctly by each call.  This file is collected last on purpose."""
import numpy as np
import pytest

import oracle as O
from paper_2008_11476_gb300 import graphs as PG
from paper_2008_11476_gb300 import hvx as H
from paper_2008_11476_gb300 import synth

pytestmark = pytest.mark.gpu

B_ORC = {H.HVX_BORDER_UNDEFINED: O.BORDER_UNDEFINED, H.HVX_BORDER_REPLICATE: O.BORDER_REPLICATE,
         H.HVX_BORDER_CONSTANT: O.BORDER_CONSTANT}
BORDERS = [H.HVX_BORDER_REPLICATE, H.HVX_BORDER_UNDEFINED, H.HVX_BORDER_CONSTANT]


def _one_call(ctx, imgs, border):
    """hvxEdgeBatchNoAlloc on `imgs` after every output was overwritten with
    7s; its outputs against hvxProcessGraphBatch's and the oracle's."""
    graphs, ref_imgs, frames, outs = [], [], [], []
    for img in imgs:
        h, w = img.shape
        inp = PG.upload(ctx, img, H.HVX_DF_U8)
        ph, mk = PG.empty(ctx, w, h, H.HVX_DF_U8), PG.empty(ctx, w, h, H.HVX_DF_U8)
        graphs.append(PG.edge_graph(ctx, inp, ph, mk, border=border, cval=0, thr=100))
        ref_imgs.append((ph, mk))
        ph2, mk2 = PG.empty(ctx, w, h, H.HVX_DF_U8), PG.empty(ctx, w, h, H.HVX_DF_U8)
        z = np.full((h, w), 7, np.uint8)  # stale values must not survive into the check
        for o in (ph2, mk2):
            H.hvxCopyImage(o, z.ctypes.data, z.strides[0], H.HVX_WRITE)
        ip, ipitch = H.hvxGetImageDevicePtr(inp)
        pp, ppitch = H.hvxGetImageDevicePtr(ph2)
        mp, mpitch = H.hvxGetImageDevicePtr(mk2)
        frames.append(H.hvx_edge_frame(ip, ipitch, pp, ppitch, mp, mpitch, w, h))
        outs.append((ph2, mk2))
    H.hvxProcessGraphBatch(graphs)
    H.hvxWaitBatch(ctx)
    H.hvxEdgeBatchNoAlloc(frames, border, 100)
    for i, (img, (a, b), (ra, rb)) in enumerate(zip(imgs, outs, ref_imgs)):
        rp, rm = PG.download(ra), PG.download(rb)
        np.testing.assert_array_equal(PG.download(a), rp, err_msg=f"phase, frame {i}")
        np.testing.assert_array_equal(PG.download(b), rm, err_msg=f"mask, frame {i}")
        op, om = O.edge_graph(img, B_ORC[border], 0, O.ROUND_ZERO, 100)
        np.testing.assert_array_equal(rp, op, err_msg=f"oracle phase, frame {i}")
        np.testing.assert_array_equal(rm, om, err_msg=f"oracle mask, frame {i}")


@pytest.mark.parametrize("k", range(len(BORDERS)))
def test_no_alloc_batch_equals_graph_batch_twice(k):
    ctx = H.hvxCreateContext()
    try:
        sizes = synth.batch_sizes(7, seed=11 + k, wlo=1, whi=900, hlo=1, hhi=500)
        sizes += [(1920, 1080), (2, 3)]
        imgs = [synth.rects_noise(w, h, seed=300 + i) for i, (w, h) in enumerate(sizes)]
        # first call: nine frames under one border
        _one_call(ctx, imgs, BORDERS[k])
        # second call: fewer frames in reverse order plus a new size, under
        # another border (different tile tables, parameters and tensor maps)
        second = imgs[::-2] + [synth.rects_noise(333, 129, seed=399)]
        _one_call(ctx, second, BORDERS[(k + 1) % len(BORDERS)])
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
