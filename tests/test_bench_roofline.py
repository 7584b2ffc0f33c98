"""The bench line's roofline arithmetic (host logic, no GPU): the radix pass
count of the view-segmented tile sort, the binning kernels' algorithmic bytes,
and the integration kernels' FP32 / MUFU fractions against the SM count and
clock, recomputed here from their definitions."""
import math

import pytest

import bench


def test_sort_passes_view_segments():
    # cone-beam C2: 180 views of 16 x 16 tiles on 256 x 256 -> 256 tiles per
    # view: 8 + 8 bits -> 2 passes (3 over the tile ids of all 180 views)
    assert bench.sort_passes(180 * 256, 180) == 2
    # PET C3: 288 views x 21 x 4 tiles -> 84 per view (7 bits) -> 2 passes
    assert bench.sort_passes(288 * 84, 288) == 2
    # fully 3-D PET: 3,168 views x 42 tiles (6 bits) -> 2 passes (4 over all tiles)
    assert bench.sort_passes(3168 * 42, 3168) == 2
    # one view of 2,048 tiles: 11 + 8 bits -> 3 passes
    assert bench.sort_passes(2048, 1) == 3
    # view << bits past 24 bits: the tile id of all views, ceil(log2 T) + 8 bits
    nv, tpv = 1 << 20, 64
    assert bench.sort_passes(nv * tpv, nv) == (26 + 8 + 7) // 8


def test_binning_bytes():
    parts = bench.binning_bytes(n_gauss=1000, n_views=10, keys=5000, tiles=10 * 256)
    e = 1000 * 10
    assert parts["k_cull"] == 60 * e
    assert parts["scan"] == 8 * e
    assert parts["k_emit"] == 16 * e + 8 * 5000
    assert parts["radix_sort"] == 16 * 2 * 5000
    assert parts["k_ranges"] == 4 * 5000 + 8 * 10 * 256


def _kernels(steps, fwd_ms, adj_ms, bin_ms):
    k = {"k_forward": {"launches": steps, "ms": fwd_ms * steps},
         "k_adjoint": {"launches": steps, "ms": adj_ms * steps}}
    for name in ("k_cull", "scan", "k_emit", "radix_sort", "k_ranges"):
        k[name] = {"launches": steps, "ms": bin_ms * steps}
    return k


@pytest.mark.parametrize("n_tof", [0, 13])
def test_roofline_fractions(monkeypatch, n_tof):
    steps, pairs = 4, 3.95e9
    monkeypatch.setattr(bench, "STEPS_TIMED", [steps])
    peaks = {"hbm_gbs": 6776.6, "source": "test", "sm_max_mhz": 2070.0}
    n_sm, mhz = 152, 2070.0
    r = bench.roofline(_kernels(steps, 7.7, 9.2, 0.2), pairs, keys=5.36e7, n_gauss=50_000, n_views=180,
                       tiles=180 * 256, n_sm=n_sm, sm_mhz=mhz, clock_note="test", peaks=peaks,
                       workload="c2", traffic_table=None, n_tof=n_tof)
    fp32_peak = n_sm * 128 * mhz * 1e6 / 1e12
    mufu_peak = n_sm * 16 * mhz * 1e6 / 1e12
    ops_f = 39.0 + 4.0 * n_tof
    ops_a = 97.5 + 8.0 * n_tof
    mufu = 3.0 + n_tof
    assert r["forward"]["peak"] == pytest.approx(fp32_peak)
    assert r["forward"]["frac"] == pytest.approx(pairs * ops_f / 7.7e-3 / 1e12 / fp32_peak)
    assert r["adjoint"]["frac"] == pytest.approx(pairs * ops_a / 9.2e-3 / 1e12 / fp32_peak)
    assert r["adjoint"]["sfu"]["frac"] == pytest.approx(pairs * mufu / 9.2e-3 / 1e12 / mufu_peak)
    # the top-level figures are the slower (dominant) kernel's
    assert r["kernel"] == "k_adjoint"
    assert r["frac"] == r["adjoint"]["frac"]
    # binning: algorithmic bytes over the five kernels' time per step
    tot = sum(bench.binning_bytes(50_000, 180, 5.36e7, 180 * 256).values())
    assert r["binning_hbm"]["bytes_per_step"] == pytest.approx(tot)
    assert r["binning_hbm"]["frac"] == pytest.approx(tot / (5 * 0.2e-3) / 1e9 / 6776.6)


def test_roofline_traffic_only_for_the_measured_sources(monkeypatch):
    monkeypatch.setattr(bench, "STEPS_TIMED", [1])
    peaks = {"hbm_gbs": 6776.6, "source": "test", "sm_max_mhz": 2070.0}
    digest = bench.sources_digest()
    args = (_kernels(1, 7.7, 9.2, 0.2), 1e9, 1e7, 1000, 10, 2560, 152, 2070.0, "test", peaks, "c2")
    good = {("c2", "k_adjoint"): (276e6, digest), ("c2", "k_forward"): (262e6, digest)}
    r = bench.roofline(*args, traffic_table=good)
    assert r["traffic"] == 276e6 and r["forward"]["traffic"] == 262e6
    stale = {("c2", "k_adjoint"): (276e6, "0" * 16)}
    assert bench.roofline(*args, traffic_table=stale)["traffic"] is None
    assert bench.roofline(*args, traffic_table={})["traffic"] is None


def test_traffic_table_matches_the_kernel_sources():
    """Every traffic entry names the digest of the sources it was measured on;
    entries for other sources are reported as null, never as this run's."""
    for (wl, kern), (bytes_, dig) in bench.TRAFFIC.items():
        assert kern in ("k_forward", "k_adjoint") and wl in bench.WORKLOADS
        assert bytes_ > 0 and len(dig) == 16
        assert math.isfinite(bytes_)
