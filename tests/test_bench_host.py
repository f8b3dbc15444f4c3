"""Host-side logic of bench.py that needs no GPU."""
import importlib.util
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    argv = sys.argv
    try:
        sys.argv = ["bench.py"]
        spec.loader.exec_module(m)
    finally:
        sys.argv = argv
    return m


def test_code_only_ignores_comments_not_code():
    b = _bench()
    src = 'int a = 1;  // one\n/* block\n comment */\nconst char* s = "// not a comment";\n\nint b = a;\n'
    out = b.code_only(src)
    assert "one" not in out and "block" not in out
    assert '"// not a comment"' in out and "int b = a;" in out
    assert b.code_only(src.replace("// one", "// uno")) == out
    assert b.code_only(src.replace("a = 1", "a = 2")) != out


def test_recorded_traffic_follows_the_kernel_code(tmp_path, monkeypatch):
    import json
    import shutil
    b = _bench()
    for rel in b.KERNEL_SOURCES["simt"]:
        os.makedirs(tmp_path / os.path.dirname(rel), exist_ok=True)
        shutil.copy(os.path.join(ROOT, rel), tmp_path / rel)
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    os.makedirs(tmp_path / "profiles")
    entry = {"engine": "simt", "source_sha": b.kernel_source_hash("simt"), "bytes_per_launch": 123}
    with open(tmp_path / "profiles" / "traffic.json", "w") as f:
        json.dump({"highdim_fp32:f32": entry}, f)
    assert b.recorded_traffic("highdim_fp32", "f32", "simt") == 123
    assert b.recorded_traffic("highdim_fp32", "bf16", "simt") is None      # other X storage
    assert b.recorded_traffic("highdim_fp32", "f32", "tcgen05") is None    # other engine
    k = tmp_path / b.KERNEL_SOURCES["simt"][0]
    k.write_text(k.read_text() + "\n// a comment\n")
    assert b.recorded_traffic("highdim_fp32", "f32", "simt") == 123        # comments do not count
    k.write_text(k.read_text() + "\nstatic int changed_code = 1;\n")
    assert b.recorded_traffic("highdim_fp32", "f32", "simt") is None       # code changed since capture


def test_reference_arm_sweep_line():
    """The oracle's side of the Table 1 sweep prints one contract line (CPU only)."""
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "sweep",
                        "--sweep-limit", "3"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def test_mean_z_separates_equal_from_shifted_posteriors():
    """The equal-accuracy statistic of the ESS block on AR(1) draws (known
    autocorrelation): two runs of one stationary process stay within 3 combined
    MCSE on nearly every coordinate, while a shift of 10 MCSE is flagged on every
    one; chain-split and half-split controls take the same statistic."""
    import numpy as np
    b = _bench()
    rng = np.random.default_rng(5)

    def ar1(n, chains, m, phi=0.8):
        x = np.zeros((n, chains, m))
        x[0] = rng.standard_normal((chains, m))
        e = rng.standard_normal((n, chains, m))
        for t in range(1, n):
            x[t] = phi * x[t - 1] + np.sqrt(1 - phi ** 2) * e[t]
        return x

    a, c = ar1(2000, 4, 3000), ar1(2000, 4, 3000)
    z = b._mean_z(a, c)
    s = b._zsum(z)
    assert z.shape == (3000,) and s["frac_above_3"] <= 0.01 and s["max_z"] < 5.0
    # the MCSE of a mean of 8000 draws with tau = (1 + phi) / (1 - phi) = 9 is about sqrt(9 / 8000)
    shift = 10 * np.sqrt(2 * 9 / 8000)
    assert b._zsum(b._mean_z(a, c + shift))["frac_above_3"] >= 0.99
    # controls: two chain groups of one run, and its two halves
    assert b._zsum(b._mean_z(a[:, :2], a[:, 2:]))["frac_above_3"] <= 0.02
    assert b._zsum(b._mean_z(a[:1000], a[1000:]))["frac_above_3"] <= 0.02
