"""The arc vs raw sampling study end to end on the GPU (fewer angles and
steps than the bench run): the raw and the arc-corrected reconstructions
place every point source within a millimetre of its centre with a finite,
few-millimetre FWHM; raw data taken for arc-corrected moves the source at
20 cm outwards."""
import math

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def test_point_source_study(torch):
    import bench
    from paper_2602_01057_gb300 import build, rgrt
    build.build()
    ctx = rgrt.Context(0)
    try:
        res = bench.point_source_study(rgrt, ctx, iters=400, n_angles=96)
    finally:
        ctx.close()
    # the mis-modelled reconstruction moves the outer sources outwards
    assert res["raw_as_arc"]["sources"][2]["peak_offset_mm"][1] > 1.5
    for mode in ("raw", "arc"):
        assert len(res[mode]["sources"]) == 3
        for src in res[mode]["sources"]:
            assert math.hypot(*src["peak_offset_mm"]) < 1.0, (mode, src)
            assert src["peak"] > 0
            for k in ("fwhm_x_mm", "fwhm_y_mm"):
                assert 0.5 < src[k] < 8.0, (mode, k, src)
