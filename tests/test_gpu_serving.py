"""Continuous batching: jobs admitted while others are running join the next
batched launch, and every job's result is bit-identical to the same job run
alone."""

import numpy as np
import pytest

from harness import scenes
from paper_2305_07083_gb300 import dfb as D
from paper_2305_07083_gb300 import serving as S

pytestmark = pytest.mark.gpu


def small_templates():
    import torch
    dev = torch.device("cuda")
    out = {"blend": [], "accumulate": []}
    for i, (W, H, g) in enumerate([(256, 256, 3), (384, 256, 4)]):
        cam = scenes.orbit_camera(W, H, 40 + i, radius=1.0)
        tid, key, rgba, depth = scenes.brick_scene_torch(W, H, 32, scenes.brick_grid((g, g, g)),
                                                         cam, 40 + i, dev)
        out["blend"].append((W, H, g ** 3, {"tile_ids": tid, "keys": key, "rgba": rgba.half(),
                                             "depth": depth,
                                             "fragment_pixels": len(tid) * 32 * 32}))
    gen = torch.Generator(device=dev)
    passes = []
    nt = 4 * 4
    for f in range(3):
        gen.manual_seed(90 + f)
        rgb = torch.rand((nt, 32 * 32, 3), generator=gen, device=dev)
        rgba = torch.cat([rgb, torch.ones((nt, 32 * 32, 1), device=dev)], -1).half()
        passes.append({"tile_ids": np.arange(nt, dtype=np.int32), "keys": np.zeros(nt, np.float32),
                       "rgba": rgba, "depth": torch.ones((nt, 32 * 32), device=dev),
                       "fragment_pixels": nt * 32 * 32})
    out["accumulate"].append((128, 128, passes))
    return out


def test_mix_equals_alone_under_continuous_batching():
    tpl = small_templates()
    arrivals = [(0.0005 * (i // 3), i % 4) for i in range(15)]     # three at a time
    jobs = S.make_jobs(tpl, arrivals, seed=3, accumulate_frames=5, T=32)
    kinds = {j.kind for j in jobs}
    assert kinds == {"blend", "accumulate"}
    # two slots for three simultaneous arrivals force queueing; the budget
    # never blocks a lone job
    budget = 3 * max(j.footprint(D.DFB_F16) for j in jobs)
    srv = S.Server(budget, max_slots=2, dtype=D.DFB_F16)
    st = srv.run(jobs)
    srv.close()
    summ = st.summary()
    assert summ["jobs"] == len(jobs)
    assert summ["max_batch"] > 1                     # jobs shared launches
    by_kind = summ["latency_ms_by_kind"]
    assert sorted(by_kind) == ["accumulate", "blend"]
    assert sum(v["jobs"] for v in by_kind.values()) == len(jobs)
    assert any(j.admitted > j.arrival for j in jobs)  # some had to wait for room
    for j in jobs:
        mixed = j.result
        fresh = S.Job(j.job_id, j.client, j.arrival, j.kind, j.W, j.H, j.T, j.frames, j.n_frames)
        alone = S.run_alone(fresh, D.DFB_F16)
        np.testing.assert_array_equal(mixed, alone)
