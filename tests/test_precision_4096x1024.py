"""Precision form of the workload: 4096x1024, 128 bricks (8x4x4), fragment
tiles stored as FP16 / BF16 / FP8 e4m3 (one FP32 scale per tile) and blended
and accumulated in FP32.  Reports, per channel, the max-abs and RMS error of
the GPU result against the FP64 oracle:

* kernel error:  oracle fed the same stored (dequantised) values;
* storage error: oracle fed the original FP32 values;

next to the fragment bytes each storage form moves.  Run with ``-s`` to see
the report line (prefixed ``PRECISION``)."""

import json

import numpy as np
import pytest

from harness import scenes
from oracle import dfb_oracle as o
from paper_2305_07083_gb300 import dfb as D

from tests.gpu_helpers import composite_once

pytestmark = pytest.mark.gpu

FORMS = [("f32", D.DFB_F32), ("f16", D.DFB_F16), ("bf16", D.DFB_BF16), ("fp8e4m3", D.DFB_FP8E4M3)]
# (kernel max-abs, storage max-abs, storage RMS) bounds; see test_gpu_parity
BOUNDS = {"f32": (1e-5, 1e-5, 1e-5), "f16": (1e-5, 2e-3, 2e-3), "bf16": (1e-5, 5e-3, 2e-3),
          "fp8e4m3": (1e-5, 8e-2, 2e-2)}


def _chan(err):
    e = err.reshape(-1, 4)
    return ([float(v) for v in np.max(np.abs(e), axis=0)],
            [float(v) for v in np.sqrt(np.mean(e ** 2, axis=0))])


def test_precision_report_4096x1024():
    sc = scenes.scene_4096x1024(seed=0)
    ref32 = o.composite_frame(sc.W, sc.H, sc.T, o.BLEND_DEPTH, sc.tile_ids, sc.keys,
                              sc.rgba.astype(np.float64), sc.depth)
    report = {"workload": "4096x1024, 64x64 tiles, 128 bricks (8x4x4), BLEND_DEPTH",
              "fragments": sc.n, "fragment_pixels": sc.fragment_pixels(), "forms": {}}
    for name, dt in FORMS:
        stored, scales = scenes.store_rgba(sc.rgba, dt)
        fb = composite_once(sc, D.DFB_BLEND_DEPTH, rgba_stored=stored, dtype=dt, scales=scales)
        got = fb.color().astype(np.float64)
        same = o.composite_frame(sc.W, sc.H, sc.T, o.BLEND_DEPTH, sc.tile_ids, sc.keys,
                                 o.dequantize(stored, dt, scales), sc.depth)
        kmax, krms = _chan(got - same)
        smax, srms = _chan(got - ref32)
        st = fb.stats()
        report["forms"][name] = {
            "bytes_per_fragment_pixel": 4 * D.ELEMENT_BYTES[dt] + 4,
            "fragment_bytes": st["fragment_bytes"],
            "kernel_max_abs_rgba": kmax, "kernel_rms_rgba": krms,
            "storage_max_abs_rgba": smax, "storage_rms_rgba": srms}
        fb.close()
    print("PRECISION " + json.dumps(report))
    for name, r in report["forms"].items():
        kb, sb, rb = BOUNDS[name]
        assert max(r["kernel_max_abs_rgba"]) <= kb, name
        assert max(r["storage_max_abs_rgba"]) <= sb, name
        assert max(r["storage_rms_rgba"]) <= rb, name
