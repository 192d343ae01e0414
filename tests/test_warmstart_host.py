"""Host-side evaluation of the learned warm start, on the CPU: the per-scan
threshold bookkeeping (scans reaching each HU threshold, mean iterations and
seconds) and the paired comparison over the scans both starts reach, on
hand-made curves whose answers are worked out below; and the scan family's
seeding."""
import numpy as np
import pytest

from paper_1402_4381_gb300 import warmstart as WS


def _rows():
    # three scans; reached[th] = (iteration, seconds)
    fbp = [dict(curve=[30.0, 15.0, 8.0], reached={20.0: (1, 0.2), 10.0: (2, 0.3)}),
           dict(curve=[25.0, 12.0, 11.0], reached={20.0: (1, 0.25)}),
           dict(curve=[40.0, 30.0, 21.0], reached={})]
    cnn = [dict(curve=[18.0, 9.0, 4.0], reached={20.0: (0, 0.05), 10.0: (1, 0.15), 5.0: (2, 0.25)}),
           dict(curve=[19.0, 9.5, 8.0], reached={20.0: (0, 0.06), 10.0: (1, 0.16)}),
           dict(curve=[35.0, 22.0, 19.0], reached={20.0: (2, 0.3)})]
    return fbp, cnn


def test_summarize_counts_and_means():
    fbp, _ = _rows()
    s = WS.summarize(fbp, thresholds=(20.0, 10.0, 5.0))
    assert s["rmsd_hu_mean_by_iteration"] == pytest.approx([95.0 / 3, 57.0 / 3, 40.0 / 3], abs=1e-3)
    t20 = s["thresholds"]["20"]
    assert (t20["reached"], t20["of"]) == (2, 3)
    assert t20["mean_iterations"] == pytest.approx(1.0)
    assert t20["mean_seconds"] == pytest.approx(0.225)
    assert s["thresholds"]["10"]["reached"] == 1 and s["thresholds"]["10"]["mean_seconds"] == pytest.approx(0.3)
    assert s["thresholds"]["5"] == {"reached": 0, "of": 3, "mean_iterations": None, "mean_seconds": None}


def test_paired_gain_uses_scans_both_starts_reach():
    fbp, cnn = _rows()
    p = WS.paired_gain(fbp, cnn, thresholds=(20.0, 10.0, 5.0))
    # 20 HU: scans 0 and 1 from both starts (scan 2 only from the network)
    assert (p["20"]["scans_both"], p["20"]["scans_only_cnn"]) == (2, 1)
    assert p["20"]["iterations_fbp"] == pytest.approx(1.0) and p["20"]["iterations_cnn"] == pytest.approx(0.0)
    assert p["20"]["seconds_fbp"] == pytest.approx(0.225) and p["20"]["seconds_cnn"] == pytest.approx(0.055)
    # 10 HU: scan 0 from both, scan 1 only from the network
    assert (p["10"]["scans_both"], p["10"]["scans_only_cnn"]) == (1, 1)
    assert p["10"]["iterations_fbp"] == pytest.approx(2.0) and p["10"]["iterations_cnn"] == pytest.approx(1.0)
    # 5 HU: only the network, on scan 0
    assert (p["5"]["scans_both"], p["5"]["scans_only_cnn"]) == (0, 1)
    assert p["5"]["iterations_fbp"] is None and p["5"]["seconds_cnn"] is None


def test_scan_family_is_seeded_and_distinct():
    base = WS.base_workload(nx=64, nviews=96, ns=111, M=6)
    a, b, a2 = WS.scan_workload(3, base), WS.scan_workload(4, base), WS.scan_workload(3, base)
    assert a == a2
    assert a.phantom_seed != b.phantom_seed and a.noise_seed != b.noise_seed
    assert 2e4 <= a.I0 <= 2e5 and a.I0 != b.I0
