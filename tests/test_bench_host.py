"""Host logic of bench.py that needs no GPU: the algorithmic work per kernel
group (the roofline numerators), the traffic record's source check, and the
workload description both arms print."""

import json
import os

import bench


class _S:
    n_beads = 32768


def test_group_work_formulas():
    prm = {"grid": 144}
    st = {"n_pairs": 5_490_000}
    n = 144
    bound, work, unit = bench.group_work("fft_green", _S(), prm, st)
    assert bound == "hbm" and unit == "GB/s"
    assert work == 4 * 6 * n * n * (n + 2) * 4  # one read and write per 3D transform, fwd + inv
    bound, work, _ = bench.group_work("spread", _S(), prm, st)
    assert work == 6 * n ** 3 * 4 + 32768 * (12 * 8 + 4 * 4)
    bound, work, unit = bench.group_work("realspace", _S(), prm, st)
    assert bound == "alu" and unit == "TFLOP/s" and work == 5_490_000 * bench.FLOP_PER_PAIR
    assert bench.group_work("krylov", _S(), prm, st)[1] is None


def test_traffic_record_matches_current_sources(tmp_path, monkeypatch):
    import hashlib

    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    for g, e in rec.items():
        h = hashlib.sha256(open(os.path.join(bench.ROOT, e["source"]), "rb").read()).hexdigest()[:16]
        want = e["bytes_per_launch"] if h == e["source_sha256_16"] else None
        assert bench.traffic_for(g) == want
    # a record taken on other sources is not used
    fake = dict(rec)
    fake["spread"] = dict(rec["spread"], source_sha256_16="0" * 16)
    (tmp_path / "profiles").mkdir()
    json.dump(fake, open(tmp_path / "profiles" / "traffic.json", "w"))
    os.makedirs(tmp_path / "paper_2607_25161_gb300" / "csrc")
    for g, e in rec.items():
        src = os.path.join(bench.ROOT, e["source"])
        dst = tmp_path / e["source"]
        dst.write_bytes(open(src, "rb").read())
    for g, e in rec.items():  # the copied sources match the (faked) record's hashes
        if g != "spread":
            fake[g] = dict(e, source_sha256_16=hashlib.sha256(
                open(os.path.join(bench.ROOT, e["source"]), "rb").read()).hexdigest()[:16])
    json.dump(fake, open(tmp_path / "profiles" / "traffic.json", "w"))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_for("spread") is None
    assert bench.traffic_for("fft_green") == rec["fft_green"]["bytes_per_launch"]


def test_group_roofline_uses_the_measured_peaks():
    prm = {"grid": 144}
    st = {"n_pairs": 5_490_000}
    pk = {"hbm_gbs": 6789.0}
    r = bench.group_roofline("fft_green", 0.2, _S(), prm, st, pk, "measured", 70e12)
    work = 4 * 6 * 144 * 144 * 146 * 4
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert abs(r["achieved"] - work / 0.2e-3 / 1e9) < 1e-6
    assert abs(r["frac"] - r["achieved"] / 6789.0) < 1e-12
    r = bench.group_roofline("realspace", 0.1, _S(), prm, st, pk, "measured", 70e12)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s" and r["peak"] == 70.0
    assert abs(r["frac"] - 5_490_000 * bench.FLOP_PER_PAIR / 0.1e-3 / 70e12) < 1e-12


def test_workload_name_is_the_benchmark_configuration():
    name = bench.workload_name(bench.WORKLOAD)
    assert name.startswith("32768 beads: 4096 rigid 8-bead")
    assert "phi 0.20" in name and "GMRES 1e-06" in name
