"""bench.py's host-side helpers: the factor-code hash ignores comments and
blank lines but not code, the committed traffic profile is used only while
that hash matches, the kernel mix reads hylu_info's flop split, and the
host accuracy metrics agree with dense arithmetic."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _hash_of(src, tmp_path, monkeypatch):
    d = tmp_path / "paper_2509_07690_gb300" / "csrc"
    d.mkdir(parents=True)
    (d / "kernels.cu").write_text(src)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return bench.kernel_hash()


SRC = """int a = 1;
// -------------------------------------------------------------- solve
int b = 2;
int launch_factor(int x) {
    return x;
}
"""


def test_factor_hash_ignores_comments_not_code(tmp_path, monkeypatch):
    h0 = _hash_of(SRC, tmp_path / "a", monkeypatch)
    h1 = _hash_of(SRC.replace("int a = 1;", "// note\nint a = 1;  // one\n\n"), tmp_path / "b", monkeypatch)
    h2 = _hash_of(SRC.replace("int a = 1;", "int a = 2;"), tmp_path / "c", monkeypatch)
    h3 = _hash_of(SRC.replace("int b = 2;", "int b = 3;"), tmp_path / "d", monkeypatch)
    assert h0 == h1                 # comments and blank lines do not count
    assert h0 != h2                 # factor code does
    assert h0 == h3                 # the substitution section does not


def test_traffic_only_with_matching_hash(tmp_path, monkeypatch):
    h = _hash_of(SRC, tmp_path, monkeypatch)
    prof = tmp_path / "profiles"
    prof.mkdir()
    f = prof / "factor_kernel_w.txt"
    f.write_text(f"# c\nfactor_source_sha256_16: {h}\ndram_bytes_per_launch: 123\n")
    assert bench.profiled_traffic("w") == 123.0
    f.write_text("factor_source_sha256_16: 0000000000000000\ndram_bytes_per_launch: 123\n")
    assert bench.profiled_traffic("w") is None
    assert bench.profiled_traffic("absent") is None


def test_measured_hbm_peak_read_or_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_hbm_gbs() == 6800.0
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6787.6}')
    assert bench.measured_hbm_gbs() == 6787.6


def test_kernel_mix_shares_sum_to_one():
    from paper_2509_07690_gb300 import Solver, synth
    A = synth.convdiff3d(10)
    s = Solver(A.n, A.rowptr, A.col, A.val, ordering=1)
    mix = bench.kernel_mix(s.info)
    assert set(mix) == {"row_row", "sup_row", "sup_sup", "in_supernode"}
    assert abs(sum(mix.values()) - 1.0) < 1e-3 and mix["sup_sup"] > 0.5
    s.close()
    e = Solver(0, [0], [], [])
    assert sum(bench.kernel_mix(e.info).values()) == 0.0
    e.close()


def test_accuracy_metrics_match_dense_arithmetic():
    """backward_error and the paper's residual ||Ax - b||_1 / ||b||_1 (Sec. 3.3)
    against the same quantities from a dense matrix."""
    import numpy as np
    from paper_2509_07690_gb300 import synth
    A = synth.circuit(300, seed=9)
    a = A.todense()
    rng = np.random.default_rng(1)
    x = rng.standard_normal(A.n)
    b = a @ x + 1e-9 * rng.standard_normal(A.n)
    r = b - a @ x
    want_be = np.abs(r).max() / (np.abs(a).sum(axis=1).max() * np.abs(x).max() + np.abs(b).max())
    want_r1 = np.abs(r).sum() / np.abs(b).sum()
    assert abs(bench.backward_error(A, A.val, x, b) - want_be) <= 1e-6 * want_be
    assert abs(bench.residual_1(A, A.val, x, b) - want_r1) <= 1e-6 * want_r1
    assert bench.residual_1(A, A.val, x, a @ x) <= 1e-14


def test_clock_samplers_are_tracked_until_stopped(tmp_path):
    """A sampler registers itself and leaves the registry when stopped, so a
    measurement abandoned half way can stop the ones it started."""
    c = bench.Clocks(0, str(tmp_path / "clocks.csv"))
    assert c in bench._ACTIVE_CLOCKS
    c.stop()
    assert c not in bench._ACTIVE_CLOCKS
    c.stop()                                  # stopping twice is harmless


def test_ordering_choice_from_the_trial():
    """Nested dissection unless its trial failed or a passing AMD trial was faster."""
    good = lambda ms: {"factor_ms": ms, "backward_error": 1e-16}   # noqa: E731
    assert bench.choose_ordering({"ND": good(50.0), "AMD": good(200.0)}) == 1
    assert bench.choose_ordering({"ND": good(250.0), "AMD": good(200.0)}) == 0
    assert bench.choose_ordering({"ND": {"error": "HyluError"}, "AMD": good(200.0)}) == 0
    assert bench.choose_ordering({"ND": {"factor_ms": 50.0, "backward_error": 1e-9}, "AMD": good(200.0)}) == 0
    assert bench.choose_ordering({"ND": good(50.0), "AMD": {"error": "HyluError"}}) == 1
    assert bench.choose_ordering({"ND": good(250.0), "AMD": {"factor_ms": 10.0, "backward_error": 1.0}}) == 1


def test_workload_orderings():
    """AMD for the 5-point grid (its configuration names AMD) and the circuit
    matrices (the configuration names AMD; nested dissection measured slower
    on the GPU), nested dissection for the PDE workloads."""
    for w in ("grid5_64", "circuit_100k", "circuit"):
        assert bench.ordering_for(w) == 0
    for w in ("convdiff3d_64", "aniso9_512"):
        assert bench.ordering_for(w) == 1


def test_default_workload_is_the_largest_single_gpu_configuration():
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--help"], capture_output=True,
                         text=True, check=True).stdout
    assert "convdiff3d_64 is the largest" in out
    assert bench.WORKLOAD == "convdiff3d_64"


def test_oracle_samples_follow_the_workload_generator(monkeypatch):
    """The CPU baseline and the reference arm sample a smaller instance of the
    timed workload's own generator (grid side or circuit size scaled)."""
    from paper_2509_07690_gb300 import synth
    monkeypatch.setattr(bench, "WORKLOAD", "convdiff3d_64")
    A = bench.sample_instance(0.25)
    B = synth.convdiff3d(16, seed=1002)
    assert A.n == 16 ** 3 and np.array_equal(A.val, B.val)
    monkeypatch.setattr(bench, "WORKLOAD", "circuit_100k")
    C = bench.sample_instance(0.1)
    D = synth.circuit(10_000, seed=1001)
    assert C.n == 10_000 and np.array_equal(C.col, D.col)
