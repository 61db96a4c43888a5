"""bench.py's reference arm (the CPU oracle timed on the host, the only arm
that runs without a GPU) prints one JSON line with the keys the driver reads;
checked here on a small grid."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--grid", "10",
                        "--steps", "2", "--warmup", "1"], capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "iters/s"
    assert d["metric"] == "reproducible PBiCGStab iters/s" and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1 and d["ms_per_step"] > 0
    assert d["scaling"] == "weak" and d["vs_baseline"] is None and d["dtype"] == "f64"
    assert d["data"] == "synthetic" and "10^3" in d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == (os.cpu_count() or 1) and cb["value"] == d["value"]
    assert "10^3" in cb["sample"] and cb["cpu"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_roofline_follows_from_its_inputs():
    """The roofline's achieved GB/s and fraction are the algorithmic bytes per
    launch over the average launch time, against the peak the line names, for
    K1 + K3 together and for each kernel; the launch counts are the ones the
    library reported (launches that returned on the stop flag are left out
    by the library, not here)."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2302_04180_gb300 import gen
    A = gen.poisson3d(12)
    prof = {"k1_spmv_dot": [100, 3.0], "k3_spmv_dot2": [100, 4.0], "k4_vec_dot2": [100, 2.0],
            "vec": [200, 2.5], "setup": [1, 0.1]}
    r = bench._roofline(A, prof)
    hbm, _ = bench._peaks()
    alg = 12 * A.nnz + 32 * A.n + 8
    assert r["alg_bytes_per_launch"] == alg and r["peak"] == hbm and r["bound"] == "hbm"
    assert r["launches"] == 200
    assert abs(r["avg_launch_us"] - 35.0) < 1e-9  # (3 + 4) ms over 200 launches
    assert abs(r["achieved"] - alg / 35e-6 / 1e9) < 1e-6 * r["achieved"]
    assert abs(r["frac"] - r["achieved"] / hbm) < 1e-12
    k1, k3 = r["per_kernel"]["K1 SpMV + <r0,s>"], r["per_kernel"]["K3 SpMV + <q,y>, <y,y>"]
    assert abs(k1["avg_launch_us"] - 30.0) < 1e-9 and abs(k3["avg_launch_us"] - 40.0) < 1e-9
    assert abs(k1["frac"] - alg / 30e-6 / 1e9 / hbm) < 1e-9
    k4 = r["per_kernel"]["K4 x, r + <r0,r>, <r,r>"]
    assert k4["alg_bytes_per_launch"] == 64 * A.n and abs(k4["avg_launch_us"] - 20.0) < 1e-9
    shares = r["time_share"]
    assert abs(sum(shares.values()) - 1.0) < 1e-3 and abs(shares["k3_spmv_dot2"] - 4.0 / 11.6) < 1e-3
