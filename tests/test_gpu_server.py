"""The request server (fs_server_*) through the C ABI: every request's result
is the same when it runs alone and when it runs in a mix of concurrent
requests on several slots, the mix really overlaps on the device, and
queued requests can be cancelled."""
import numpy as np
import pytest

from paper_2409_08270_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fsb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_08270_gb300 import build, flashsplat
    build.build()
    flashsplat.load()
    return flashsplat


def _scenes():
    return [synth.tiny_scene(),
            synth.binary_scene(n=20000, views=6, width=400, height=300),
            synth.multi_scene(n=30000, views=6, width=320, height=240, n_clusters=6),
            synth.binary_scene(seed=synth.SEED_BASE + 9, n=15000, views=5, width=512, height=384)]


def _requests(scenes, k=3):
    """k requests per scene: the scene's masks with fresh seeded noise and a
    bias from the paper's grid."""
    reqs = []
    for sid, w in enumerate(scenes):
        for r in range(k):
            rng = np.random.default_rng(1000 * sid + r)
            masks = []
            for m in w.masks:
                flip = rng.random(m.shape) < 0.02
                if w.E == 2:
                    masks.append(np.where(flip, 1 - m, m).astype(m.dtype))
                else:
                    masks.append(np.where(flip, rng.integers(0, w.E, m.shape), m).astype(m.dtype))
            reqs.append((sid, masks, [0.0, 0.4, -0.4][r % 3]))
    return reqs


def _same(a, b):
    decided = (a["margin"] > 1e-9) & (b["margin"] > 1e-9)
    assert np.array_equal(a["label"][decided], b["label"][decided])
    if a["bits"] is not None:
        assert np.array_equal(a["bits"][decided], b["bits"][decided])
    fin = np.isfinite(a["margin"])
    np.testing.assert_allclose(a["margin"][fin], b["margin"][fin], rtol=1e-5, atol=1e-7)


def test_results_alone_equal_results_in_the_mix(fsb):
    scenes = _scenes()
    reqs = _requests(scenes)
    # alone: one slot, one request at a time
    solo = fsb.Server(slots=1)
    try:
        ids = [solo.add_scene(w.gaussians) for w in scenes]
        alone = []
        for sid, masks, gamma in reqs:
            t = solo.submit(ids[sid], scenes[sid].cams, masks, scenes[sid].E, gamma)
            alone.append(solo.fetch(t))
    finally:
        solo.close()
    # in the mix: three slots, everything submitted at once
    srv = fsb.Server(slots=3)
    try:
        ids = [srv.add_scene(w.gaussians) for w in scenes]
        tickets = [srv.submit(ids[sid], scenes[sid].cams, masks, scenes[sid].E, gamma)
                   for sid, masks, gamma in reqs]
        mixed = [srv.fetch(t) for t in tickets]
    finally:
        srv.close()
    for a, b in zip(alone, mixed):
        _same(a, b)
        assert b["info"].status == fsb.FS_OK and b["info"].done == 1
        assert b["info"].submit_s <= b["info"].start_s <= b["info"].done_s
    # the mix ran on several slots at once
    infos = [m["info"] for m in mixed]
    assert len({i.slot for i in infos}) >= 2
    overlaps = sum(1 for i in infos for j in infos
                   if i.slot != j.slot and i.start_s < j.done_s and j.start_s < i.done_s)
    assert overlaps > 0
    # and the solves did the same work
    for a, b in zip(alone, mixed):
        assert a["info"].stats.pairs == b["info"].stats.pairs


def test_cancel_and_bad_requests(fsb):
    w = synth.binary_scene(n=20000, views=8, width=640, height=480)
    srv = fsb.Server(slots=1)
    try:
        sid = srv.add_scene(w.gaussians)
        with pytest.raises(fsb.FlashSplatError) as ei:
            fsb.fs_server_submit(srv.srv, sid + 7, fsb.make_cameras(w.cams),
                                 [m.ctypes.data for m in w.masks], fsb.FS_U8, w.E, 0.5)
        assert ei.value.status == fsb.FS_INVALID_ARGUMENT
        tickets = [srv.submit(sid, w.cams, w.masks, w.E, 0.5) for _ in range(4)]
        srv.cancel(tickets[-1])              # still queued behind the others
        with pytest.raises(fsb.FlashSplatError) as ei:
            srv.fetch(tickets[-1])
        assert ei.value.status == fsb.FS_CANCELLED
        res = [srv.fetch(t) for t in tickets[:-1]]
        for r in res[1:]:
            _same(res[0], r)
    finally:
        srv.close()


def test_autotune_keeps_results(fsb):
    w = synth.binary_scene(n=20000, views=6, width=400, height=300)
    plain = fsb.Server(slots=1)
    tuned = fsb.Server(slots=2, autotune=True)
    try:
        a = plain.fetch(plain.submit(plain.add_scene(w.gaussians), w.cams, w.masks, w.E, 0.5))
        sid = tuned.add_scene(w.gaussians)
        b = [tuned.fetch(tuned.submit(sid, w.cams, w.masks, w.E, 0.5)) for _ in range(2)]
    finally:
        plain.close()
        tuned.close()
    for r in b:
        _same(a, r)
        assert (r["info"].views_per_batch, r["info"].depth_chunks) in \
            {(50, 6), (32, 5), (64, 6), (16, 4), (50, 4)}


def test_captured_solve_serving_equals_plain_serving(fsb):
    """graphs > 0: each scene's requests replay its captured solve with the
    request's masks written into the captured buffers (fresh noise each
    time); a request with another gamma captures the scene again.  Results
    equal one-at-a-time plain solves."""
    scenes = _scenes()[:3]
    reqs = []
    for sid, w in enumerate(scenes):
        for r in range(3):
            rng = np.random.default_rng(500 + 10 * sid + r)
            masks = []
            for m in w.masks:
                flip = rng.random(m.shape) < 0.02
                if w.E == 2:
                    masks.append(np.where(flip, 1 - m, m).astype(m.dtype))
                else:
                    masks.append(np.where(flip, rng.integers(0, w.E, m.shape), m).astype(m.dtype))
            reqs.append((sid, masks, 0.5 if r < 2 else -0.4))
    solo = fsb.Server(slots=1)
    try:
        ids = [solo.add_scene(w.gaussians) for w in scenes]
        alone = [solo.fetch(solo.submit(ids[s], scenes[s].cams, m, scenes[s].E, g))
                 for s, m, g in reqs]
    finally:
        solo.close()
    srv = fsb.Server(slots=2, graphs=2)      # fewer kept graphs than scenes: some are dropped
    try:
        ids = [srv.add_scene(w.gaussians) for w in scenes]
        tickets = [srv.submit(ids[s], scenes[s].cams, m, scenes[s].E, g) for s, m, g in reqs]
        served = [srv.fetch(t) for t in tickets]
    finally:
        srv.close()
    for a, b in zip(alone, served):
        _same(a, b)
        assert b["info"].status == fsb.FS_OK


def test_bounded_fetch_returns_timeout(fsb):
    """A fetch whose bounded wait runs out reports FS_TIMEOUT (None here) and
    leaves the request in place; a blocking fetch then returns it."""
    w = synth.binary_scene(n=200000, views=20, width=1008, height=756)
    srv = fsb.Server(slots=1)
    try:
        sid = srv.add_scene(w.gaussians)
        t = srv.submit(sid, w.cams, w.masks, w.E, 0.5)
        assert srv.fetch(t, timeout_ms=1) is None
        res = srv.fetch(t)
        assert res["info"].status == fsb.FS_OK
        assert (res["label"] >= 0).sum() > 0
    finally:
        srv.close()
