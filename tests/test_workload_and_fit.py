"""Host logic with no GPU: the workload generators' structure (batched
uneven circuits, the depth-augmented staircase) and the boundary fit used by
the paper-workload sweep."""

import math

import pytest

import bench
import workload as w


def test_uneven_batch_obeys_its_ranges():
    items = w.uneven_batch(64, 0)
    assert len(items) == 64
    for it in items:
        assert 16 <= it.q <= 26 and it.depth in (8, 16, 32)
        assert len(it.seg_sizes) in (2, 3) and sum(it.seg_sizes) == it.q
        assert min(it.seg_sizes) >= 4
        assert 2 <= sum(it.cuts_per_boundary) <= 6
        # the boundary CZs are exactly the requested cuts
        bounds, acc = [], 0
        for s in it.seg_sizes[:-1]:
            acc += s
            bounds.append(acc)
        crossing = sum(1 for g in it.gates if g.kind == "CZ" and g.q1 in bounds and g.q0 == g.q1 - 1)
        assert crossing == sum(it.cuts_per_boundary)
    assert w.uneven_batch(8, 3) == w.uneven_batch(8, 3)  # seeded


def test_staircase_depth_structure():
    q, blocks, p = 7, 3, 2
    base = w.staircase(q, blocks)
    g = w.staircase_depth(q, blocks, p)
    assert len(g) == len(base) + 2 * 10 ** p
    pad_top = g[q:q + 100]
    assert [x.kind for x in pad_top[:4]] == ["T", "X", "T", "X"]
    assert all(x.q0 == 0 for x in pad_top)
    assert all(x.q0 == q - 1 for x in g[-100:])
    assert g[:q] == base[:q] and g[q + 100:-100] == base[q:]
    # cut count unchanged: one boundary CX per block for n = 2
    cuts = sum(1 for x in g if x.kind == "CX" and x.q0 < q // 2 <= x.q1)
    assert cuts == blocks


@pytest.mark.parametrize("slope,intercept", [(0.5, 0.0), (0.7, -7.3), (1.0, -11.5)])
def test_fit_boundary_recovers_a_separating_line(slope, intercept):
    pts = [(q, c, c - (slope * q + intercept)) for q in range(2, 31, 2) for c in range(0, 15)
           if abs(c - (slope * q + intercept)) > 1e-9]
    fit = bench.fit_boundary(pts)
    # every grid point is classified as the line it was drawn from classifies it,
    # except possibly points within one grid step of the line
    for q, c, d in pts:
        side = c - (fit["slope"] * q + fit["intercept"])
        if abs(d) > 1.0:
            assert math.copysign(1, side) == math.copysign(1, d), (q, c, d, fit)


def test_fit_boundary_takes_the_upper_edge_of_a_band():
    # speedups only between a lower edge (the fewest cuts lose too, as on the
    # staircase, whose uncut time grows with its cut blocks) and the line
    # c = 0.5 q - 2; q below 12 has no speedup at all
    slope, intercept = 0.5, -2.0
    pts = []
    for q in range(4, 31, 2):
        for c in range(0, 15):
            up = c - (slope * q + intercept)
            if abs(up) < 1e-9:
                continue
            win = q >= 12 and c >= 3 and up < 0
            pts.append((q, c, -1.0 if win else 1.0))
    fit = bench.fit_boundary(pts)
    assert abs(fit["slope"] - slope) < 0.1 and abs(fit["intercept"] - intercept) < 1.5, fit


def test_fit_boundary_needs_both_classes():
    assert bench.fit_boundary([(4, 1, -0.5), (6, 2, -0.1)]) is None


def test_planner_threshold_matches_the_oracle():
    # the planner's own Eqs. 13-14 (product code) against the oracle's
    from oracle import thresholds as th
    from paper_2603_01443_gb300 import planner

    for n in (2, 3, 4, 6, 8):
        for q in range(4, 40):
            assert planner.threshold(q, n) == pytest.approx(th.threshold(q, n), abs=1e-12)
    with pytest.raises(ValueError):
        planner.threshold(10, 1)


def test_splitmix64_reference_sequence():
    # the first outputs of SplitMix64 from state 0 (Steele, Lea, Flood 2014;
    # the widely used reference sequence), and the derived doubles and angles
    r = w.SplitMix64(0)
    assert [r.next_u64() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                                0x06C45D188009454F]
    r = w.SplitMix64(0)
    assert r.next_double() == (0xE220A8397B1DCDAF >> 11) / 2.0 ** 53
    a = r.next_angle()
    assert a == 2.0 * math.pi * ((0x6E789E6AA1B965F4 >> 11) / 2.0 ** 53) and 0.0 <= a < 2 * math.pi


def test_traffic_records_follow_the_kernel_source(monkeypatch, tmp_path):
    # a DRAM-traffic record is used only for its own workload and only while
    # the kernel source it was taken on is unchanged
    import json

    csrc = tmp_path / "paper_2603_01443_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_text("// kernel v1\n")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    a = bench.parse_args([])
    rec = {"sources": ["k.cu"], "source_hash": bench.kernel_source_hash(["k.cu"]),
           "dram_bytes_per_launch": 123.0}
    (tmp_path / "profiles" / "traffic.json").write_text(
        json.dumps({bench.traffic_key("kern", a): rec}))
    assert bench.recorded_traffic("kern", a) == 123.0
    assert bench.recorded_traffic("kern", bench.parse_args(["--q", "28"])) is None
    assert bench.recorded_traffic("other", a) is None
    (csrc / "k.cu").write_text("// kernel v1 with a changed comment\n")
    assert bench.recorded_traffic("kern", a) is None


def test_fp32_peak_from_unit_counts():
    # 152 SMs x 128 FP32 lanes x 2 flops per FMA x 2070 MHz
    assert abs(bench.fp32_peak_tflops() - 80.55) < 0.01


def test_clock_samples_summary():
    # nvidia-smi CSV lines (FIELDS order): the median SM clock under load, the
    # maximum clock and each throttle reason that was Active at least once
    out = "\n".join([
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1398.7, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ])
    s = bench.ClockSampler.summarize(out)
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "samples": 3,
                 "reasons": ["sw_power_cap"]}
    hot = out + "\n0, 1500, 2070, 1400, 0x48, Not Active, Active, Not Active, Active"
    assert bench.ClockSampler.summarize(hot)["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert bench.ClockSampler.summarize("") is None


def test_planner_eq15_threshold_matches_the_oracle():
    # Eq. 15: no change at D_seg = D / n, the oracle's full reduction at D_seg = D
    from oracle import thresholds as th
    from paper_2603_01443_gb300 import planner

    for n in (2, 3, 4, 5):
        for q in (12.0, 20.0, 30.0):
            assert planner.nonuniform_threshold(q, n, 1.0 / n) == pytest.approx(th.threshold(q, n))
            assert planner.nonuniform_threshold(q, n, 1.0) == pytest.approx(
                th.threshold(q, n) - th.nonuniform_reduction(n))
            mid = planner.nonuniform_threshold(q, n, 0.5 * (1.0 / n + 1.0))
            assert th.threshold(q, n) - th.nonuniform_reduction(n) < mid < th.threshold(q, n)


def test_planner_depth_ratio():
    # brickwork: every layer touches every segment (D_seg = D); a CX ladder
    # crosses the segments one after another (D_seg near D / n)
    from paper_2603_01443_gb300 import planner

    assert planner.depth_ratio(w.brickwork(12, 6, 0), [6, 6]) == pytest.approx(1.0)
    ladder = [w.Gate("CX", i, i + 1) for i in range(11)]
    r = planner.depth_ratio(ladder, [6, 6])
    assert r == pytest.approx(6 / 11)
    assert planner.circuit_depth(ladder) == 11


def test_planner_decide_filters_forms_and_falls_back():
    # decide() with canned predictions (host logic only): forms beyond the
    # tolerance are never chosen; a large held-out error near an option
    # sends the decision to Eqs. 13-15
    import numpy as np

    from paper_2603_01443_gb300 import planner

    P = planner.StagePlanner.__new__(planner.StagePlanner)
    P.fallback_spread = P.fallback_error = 0.2
    P.hold_x = None
    opts = [{"n": 2, "form": f, "seg_tile_bits": 13, "features": [float(planner.FORMS.index(f))],
             "cut_bits": 4, "n_sub": 32} for f in ("fma", "tf32x3", "bf16x3")]
    cut = {"fma": 3.0, "tf32x3": 2.0, "bf16x3": 1.0}

    def predict(X):
        c = np.array([cut[planner.FORMS[int(x[0])]] for x in X])
        return {"cut": c, "orig": np.full(len(X), 10.0), "spread": np.zeros(len(X))}

    P.predict = predict
    P.expected_error = lambda X: np.zeros(len(X))
    assert P.decide(20, opts, tol=2e-6)["form"] == "tf32x3"
    assert P.decide(20, opts, tol=5e-5)["form"] == "bf16x3"
    P.expected_error = lambda X: np.full(len(X), 0.5)
    d = P.decide(20, opts, tol=2e-6, dseg_over_d=1.0)
    assert d["fallback"] and d["choice"] == 2 and d["form"] == "auto"  # 4 < 20/2 - 1
    d = P.decide(9, opts, tol=2e-6, dseg_over_d=1.0)
    assert d["fallback"] and d["choice"] == 0  # 4 >= 9/2 - 1
    # among admissible chains the fallback takes the fewest cuts: four
    # segments with 4 cuts per boundary (12, below Eq. 14 at q = 30) lose to
    # two segments with 4
    chain = [{"n": n, "form": "fma", "seg_tile_bits": 13, "features": [0.0],
              "cut_bits": 4 * (n - 1), "n_sub": 2 * 16 + (n - 2) * 256} for n in (4, 3, 2)]
    d = P.decide(30, chain, tol=2e-6, dseg_over_d=0.5)
    assert d["fallback"] and d["choice"] == 2
