"""Host logic of bench.py that sets the roofline and baseline figures: the
per-kernel algorithmic bytes (pruned extents, stored x columns), the
unpruned whole-map minimum B_alg, and the guard that skips the FP64 oracle
baseline where one map would not fit the host's memory."""
import bench


def test_whole_box_bytes():
    N, npix = 256, 1000
    ab = bench.algorithmic_bytes(N, npix)
    box = 4 * N ** 3
    assert ab["draw_zfft"] == box
    assert ab["yfft"] == box + box                  # read every plane, write every row
    assert ab["xc2r"] == box + box
    assert ab["gather"] == 24 * npix


def test_pruned_bytes_with_stored_columns():
    N, planes, rows, stored = 512, 190, 66166, 3594624
    ab = bench.algorithmic_bytes(N, 0, planes, rows, None, planes, stored)
    row = 4 * N
    assert ab["draw_zfft"] == 4 * N * N * planes     # only the listed planes are stored
    assert ab["yfft"] == planes * N * row + rows * row
    assert ab["xc2r"] == rows * row + 4 * stored     # whole rows read, stored reals written
    # without the stored-column count the x pass is charged whole rows both ways
    assert bench.algorithmic_bytes(N, 0, planes, rows)["xc2r"] == 2 * rows * row


def test_b_alg_is_the_unpruned_minimum():
    N, npix = 1024, 20132659
    half = 8 * N * N * (N // 2 + 1)                # complex half spectrum
    assert bench.b_alg_bytes(N, npix) == 2 * half + 4 * N ** 3 + 20 * npix
    assert bench.b_alg_bytes(N, npix) == 13304332284


def test_oracle_baseline_skipped_when_the_box_does_not_fit(monkeypatch):
    w = bench.WORKLOADS["box2048_cap0.4_learned"]
    monkeypatch.setattr(bench, "host_memory_bytes", lambda: 64 * 2 ** 30)
    cb = bench.cpu_baseline(w, type("A", (), {"workload": w.name})())
    assert cb["value"] is None and "GiB" in cb["sample"] and cb["kind"] == "oracle"


def test_reference_arm_unavailable_when_the_box_does_not_fit(monkeypatch, capsys):
    import json
    monkeypatch.setattr(bench, "host_memory_bytes", lambda: 64 * 2 ** 30)
    args = type("A", (), {"workload": "box2048_cap0.4_learned", "warmup": 1, "steps": 1, "ref_budget_s": 1.0})()
    bench.run_reference(args, 0, 1)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and "unavailable" in line
