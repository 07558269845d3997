"""The benchmark's roofline arithmetic for the two-stage reduction (host
logic, CPU only): the bulge chase is the reported kernel, its algorithmic
flops are counted from the chase's task structure, the occupied-SM fraction
and the one-stage-equivalent rate follow from the event times given, and the
DRAM traffic comes from the committed capture only while band.cu is the file
it was taken on."""
import hashlib
import importlib.util
import json
import math
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def chase_tasks(n, nb=8):
    # sweep s annihilates column s and chases its bulge down in blocks of nb:
    # ceil((n - 1 - s) / nb) tasks, counted here by brute force
    total = 0
    for s in range(n - 1):
        rows = n - 1 - s
        t = 0
        while rows > 0:
            rows -= nb
            t += 1
        total += t
    return total


def test_band_roofline_reports_the_bulge_chase():
    bench = load_bench()
    n, nk_all, nk = 882, 90, 23
    red = {"matrices": nk, "panel_qr": 40.0, "a22_v": 27.3, "w_form": 13.4,
           "rank2_update": 60.3, "bulge_chase": 38.6}
    ph = {"tridiag": 165.5}
    peaks = {"fp64_nominal_tflops": 1.25856, "sms": 152}
    roof, red_obj = bench.band_roofline(red, n, nk_all, ph, peaks)
    assert roof["kernel"].startswith("bulge_kernel") and roof["bound"] == "alu"
    assert roof["unit"] == "TFLOP/s" and roof["peak"] == peaks["fp64_nominal_tflops"]
    tasks = chase_tasks(n)
    assert tasks == 48951
    # 6 nb^2 complex multiply-adds per task, 8 real flops each
    flops = nk * tasks * 6 * 64 * 8
    achieved = flops / (red["bulge_chase"] / 1e3) / 1e12
    assert math.isclose(roof["achieved"], achieved, rel_tol=1e-12)
    assert math.isclose(roof["frac"], achieved / peaks["fp64_nominal_tflops"], rel_tol=1e-12)
    assert roof["occupied_sms"] == nk
    occ = peaks["fp64_nominal_tflops"] * nk / peaks["sms"]
    assert math.isclose(roof["frac_of_occupied_sms"], achieved / occ, rel_tol=1e-12)
    assert set(roof["group_rates"]) == {"rank2_update", "a22_v", "bulge_chase", "panel_qr",
                                        "w_form"}
    eff = nk_all * 16.0 / 3.0 * n ** 3 / (ph["tridiag"] / 1e3) / 1e12
    assert math.isclose(red_obj["one_stage_equivalent_tflops"], eff, rel_tol=1e-12)
    assert red_obj["timed_part_matrices"] == nk


def test_band_roofline_traffic_follows_the_capture():
    bench = load_bench()
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))["bulge_kernel"]
    src = os.path.join(ROOT, "paper_1310_6380_gb300", "csrc", rec["source"])
    same = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] == rec["sha256_16"]
    red = {"matrices": 23, "panel_qr": 1.0, "a22_v": 1.0, "w_form": 1.0, "rank2_update": 1.0,
           "bulge_chase": 38.6}
    roof, _ = bench.band_roofline(red, 882, 90, {"tridiag": 165.5},
                                  {"fp64_nominal_tflops": 1.25856, "sms": 152})
    if same:
        assert roof["traffic"] == rec["dram_bytes_per_matrix"] * 23
    else:
        assert roof["traffic"] is None
    # another size than the captured one has no traffic figure
    roof, _ = bench.band_roofline(dict(red), 450, 30, {"tridiag": 50.0},
                                  {"fp64_nominal_tflops": 1.25856, "sms": 152})
    assert roof["traffic"] is None
