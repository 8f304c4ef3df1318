"""Host-side logic of the serving loop: arrivals, job mix and footprints
(no GPU needed)."""

import numpy as np

from paper_2305_07083_gb300 import dfb as D
from paper_2305_07083_gb300 import serving as S


def test_poisson_arrivals_are_seeded_sorted_and_have_the_mean_gap():
    a = S.poisson_arrivals(4, 0.008, 2.0, seed=1)
    b = S.poisson_arrivals(4, 0.008, 2.0, seed=1)
    assert a == b and a == sorted(a) and {c for _, c in a} == {0, 1, 2, 3}
    gaps = np.diff([t for t, c in a if c == 0])
    assert abs(gaps.mean() - 0.008) < 0.002           # about 250 arrivals per client


def _fake_templates():
    f = {"tile_ids": np.arange(4, dtype=np.int32), "keys": np.zeros(4, np.float32),
         "rgba": None, "depth": None, "fragment_pixels": 4 * 64 * 64}
    return {"blend": [(256, 256, 8, f)], "accumulate": [(128, 128, [f, f])]}


def test_job_mix_and_footprint():
    arrivals = [(0.001 * i, i % 4) for i in range(200)]
    jobs = S.make_jobs(_fake_templates(), arrivals, seed=0, accumulate_frames=64)
    kinds = [j.kind for j in jobs]
    assert 60 < kinds.count("blend") < 140
    acc = next(j for j in jobs if j.kind == "accumulate")
    assert acc.n_frames == 64 and len(acc.frames) == 2
    # framebuffers (68 B per pixel) + the referenced fragment tiles
    fp16 = acc.footprint(D.DFB_F16)
    assert fp16 == 128 * 128 * 68 + 2 * 4 * 64 * 64 * (8 + 4)
    assert acc.footprint(D.DFB_F32) > fp16


def test_admission_order_budget_and_slots():
    fp = lambda j: j[1]
    # arrival order, budget 10: 4 + 5 fit, 3 would exceed it and stops the rest
    q = [("a", 4), ("b", 5), ("c", 3), ("d", 1)]
    got = S.admit(q, 0, 0, 10, 8, fp)
    assert [j[0] for j in got] == ["a", "b"] and [j[0] for j in q] == ["c", "d"]
    # no overtaking: "d" (1) would fit but waits behind "c"
    assert S.admit(q, 2, 9, 10, 8, fp) == [] and len(q) == 2
    # slots bound the admission even when the budget does not
    q = [("x%d" % i, 1) for i in range(6)]
    assert len(S.admit(q, 3, 0, 100, 5, fp)) == 2 and len(q) == 4
    # an idle server takes the head job even if it alone exceeds the budget
    q = [("big", 50), ("small", 1)]
    got = S.admit(q, 0, 0, 10, 8, fp)
    assert [j[0] for j in got] == ["big"] and q == [("small", 1)]
    # ... but not while anything is active
    q = [("big", 50)]
    assert S.admit(q, 1, 0, 10, 8, fp) == [] and q == [("big", 50)]


def test_summary_splits_latency_by_job_kind():
    st = S.ServerStats()
    for kind, v in [("blend", 1.0), ("blend", 3.0), ("accumulate", 40.0), ("blend", 2.0)]:
        st.latencies_ms.append(v)
        st.latencies_by_kind.setdefault(kind, []).append(v)
    summ = st.summary()
    assert summ["latency_ms_p50"] == 2.5
    assert summ["latency_ms_by_kind"]["blend"] == {"jobs": 3, "p50": 2.0,
                                                   "p99": float(np.percentile([1, 3, 2], 99))}
    assert summ["latency_ms_by_kind"]["accumulate"] == {"jobs": 1, "p50": 40.0, "p99": 40.0}
