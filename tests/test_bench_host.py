"""Host checks of the benchmark's bookkeeping (no GPU): the per-part algorithmic model, the launch
count it claims, the roofline of a synthetic per-part timing, and the kernel-code hash that keys the
stored DRAM traffic."""
import json
import os

import numpy as np

import bench


def _info(local_form=2, lag_store=1, far=1):
    return dict(W=23, nmax=32, n_pairs=4754014, n_modes=313071, n_far_modes=12000, n_kappa=40000, n_lambda=120,
                nb=608, nf=2048, kernel_width=8, n_self=10000, n_self_soe=75, lag_active=1, lag_store=lag_store,
                far_active=far, Nh=447, local_form=local_form, local_nc=16, n_near_pairs=100000, local_variant=0)


def test_part_model_covers_every_part_and_the_factored_form_moves_fewer_bytes():
    parts = {"local", "self", "ingest", "combine", "spread", "modes", "far", "interp", "fft_type1", "fft_type2"}
    stored = bench.part_model(_info(local_form=1), 10000, 10000, False)
    factored = bench.part_model(_info(local_form=2), 10000, 10000, False)
    assert set(stored) == parts and set(factored) == parts
    assert all(v["bytes"] > 0 for v in factored.values() if v is not None)
    # 32 FP32 weights + index per pair against an 8-byte record (+ near rows, y, windows)
    assert stored["local"]["bytes"] == 4754014 * (32 * 4 + 4) + 10000 * 32 * 4 + 10000 * 16
    assert factored["local"]["bytes"] < stored["local"]["bytes"] / 5
    # the recomputed lag adds a second spread and a second type-1 transform
    rec = bench.part_model(_info(lag_store=0), 10000, 10000, False)
    assert rec["fft_type1"]["bytes"] == 2 * factored["fft_type1"]["bytes"]
    assert rec["spread"]["bytes"] == 2 * factored["spread"]["bytes"]


def test_launch_count_per_step():
    # ingest, local (2 factored), self, combine, spread + transpose, modes, far, transpose, interp, tick
    assert bench.launches_per_step(_info(local_form=2), 1) == 12
    assert bench.launches_per_step(_info(local_form=1), 1) == 11
    assert bench.launches_per_step(_info(local_form=2, lag_store=0), 0) == 13
    assert bench.launches_per_step(_info(local_form=1, far=0), 0) == 9


def test_roofline_picks_the_largest_kernel_of_ours_and_bounds_it():
    info = _info()
    parts = {"local": (4.4, 100), "modes": (6.2, 100), "fft_type1": (9.0, 100), "self": (1.8, 100)}
    r = {"info": info, "parts": parts, "workload": "cfg2"}
    roof, per = bench.roofline(r, 10000, 10000, False)
    assert roof["kernel"] == "modes"  # cuFFT's parts are never the dominant kernel of ours
    m = bench.part_model(info, 10000, 10000, False)["modes"]
    assert abs(per["modes"]["GB/s"] - m["bytes"] / 62e-6 / 1e9) < 1e-6 * per["modes"]["GB/s"]
    assert roof["bound"] == per["modes"]["bound"] and 0 < roof["frac"]


def test_kernel_code_hash_ignores_comments(tmp_path, monkeypatch):
    d = tmp_path / "paper_2604_07170_gb300" / "csrc"
    d.mkdir(parents=True)
    for fn in ("wfp_step.cu", "wfp_dev.h"):
        (d / fn).write_text("int f() {  // first\n    return 1;\n}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.source_hash("modes")
    (d / "wfp_step.cu").write_text("// a comment\nint f() {  // second\n\n    return 1;\n}\n")
    assert bench.source_hash("modes") == h0
    (d / "wfp_step.cu").write_text("int f() {\n    return 2;\n}\n")
    assert bench.source_hash("modes") != h0


def test_stored_traffic_entries_match_the_current_kernel_code_or_are_reported_stale():
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as f:
        tr = json.load(f)
    for key, e in tr.items():
        kind = "local_factored" if key.endswith(":factored") else key.split(":")[0]
        assert set(e) >= {"bytes_per_launch", "dram_read", "dram_write", "source_hash", "capture", "kernel"}
        assert e["bytes_per_launch"] == e["dram_read"] + e["dram_write"]
        assert "--clock-control none" in e["capture"]
        # the bench reports the entry only while the hash matches; the stored-weight local part's
        # entries (the FP64 line's dominant kernel) must match the committed code
        if kind == "local":
            assert e["source_hash"] == bench.source_hash(kind), key


def test_grid_term_counts_the_band_or_its_written_tiles():
    # spreading writes and interpolation reads the nb x nb sub-box of the [nb][nf] band that the points
    # map to (its non-empty tiles when known)
    info = _info()
    m = bench.part_model(info, 10000, 10000, False)
    assert m["interp"]["bytes"] == 608 * 608 * 4 + 10000 * (2 * 8 * 4 + 4 + 8)
    info.update(spread_tile=16, n_spread_tiles=1000)
    m = bench.part_model(info, 10000, 10000, False)
    assert m["interp"]["bytes"] == 1000 * 256 * 4 + 10000 * (2 * 8 * 4 + 4 + 8)
    assert m["spread"]["bytes"] == 1000 * 256 * 4 + 10000 * (2 * 8 * 4 + 4 + 4)


def test_launch_count_without_the_lagged_regime():
    # no lag (T < A+): one spread, no far history
    info = _info(local_form=2)
    info.update(lag_active=0, lag_store=0)
    assert bench.launches_per_step(info, 1) == 11


def test_accuracy_of_kept_steps():
    rng = np.random.default_rng(0)
    ref = rng.standard_normal((2, 50))
    kept = np.zeros((2, 200))
    idx = rng.choice(200, 50, replace=False)
    kept[:, idx] = ref * (1 + 1e-7)
    a = bench.accuracy({"kept": kept, "kept_steps": [9, 10]}, idx, ref)
    assert abs(a["rel_l2_vs_oracle"] - 1e-7) < 1e-12 and a["targets"] == 50 and a["steps"] == [9, 10]
