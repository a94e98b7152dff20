"""Host-side arithmetic of bench.py on CPU: the connection count per configuration that the
benchmark's connections/s is built on, the algorithmic bytes of the sort kernels that enter the
roofline line, and the rule that a committed DRAM-traffic figure is used only while the kernel
source it was captured from is unchanged."""
import hashlib
import os

import pytest

import bench
from paper_2601_21310_b300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


# singles + same-spin doubles + opposite-spin doubles per configuration of the four workload
# shapes: n(norb - n) per spin, C(n,2) C(norb-n,2) per spin, (n (norb - n))^2
@pytest.mark.parametrize("name,per_det", [("tiny_n10", 875), ("small_n16", 5792),
                                          ("cr2_24e30o", 67284), ("cr2_48e42o", 271944)])
def test_connections_per_configuration(olib, name, per_det):
    wl = synth.WORKLOADS[name]
    assert bench.synth_nexc(wl) == per_det
    # the oracle's connected set (Eq. connected_set) has the same size
    assert olib.n_excitations(wl.norb, wl.nalpha, wl.nbeta) == per_det


def test_connected_set_size_matches_enumeration(olib):
    # one configuration of the 16-orbital workload, enumerated by the oracle
    wl = synth.WORKLOADS["small_n16"]
    S = synth.select_S(wl.norb, wl.nalpha, 64)
    for a, b in S[[0, 7, 63]]:
        assert len(olib.excitations(wl.norb, a, b)) == bench.synth_nexc(wl)


def test_sort_bytes_per_pair():
    # a radix pass reads and writes key + FP64 value; keys are 4 B for 2 norb <= 32, 8 B up to
    # 64, 16 B above
    n = 1_000_000
    for name, key in (("small_n16", 4), ("cr2_24e30o", 8), ("cr2_48e42o", 16)):
        wl = synth.WORKLOADS[name]
        bound, b, unit = bench.algorithmic_work("rs_scatter", wl, 1, 1, 0, n, 0, 0)
        assert (bound, unit) == ("hbm", "B") and b == 2 * (key + 8) * n
        bound, b, _ = bench.algorithmic_work("rs_hist", wl, 1, 1, 0, n, 0, 0)
        assert b == key * n
        # with B buckets a sort launch handles 1/B of the pairs
        _, b4, _ = bench.algorithmic_work("rs_scatter", wl, 1, 1, 0, n, 0, 0, buckets=4)
        assert b4 == 2 * (key + 8) * n / 4
    # issue-bound kernels carry no byte roofline
    assert bench.algorithmic_work("conn_count", synth.WORKLOADS["small_n16"], 1, 1, 0, 0, 0,
                                  0)[0] == "alu"


def _profile_fields(path):
    vals = {}
    with open(path) as f:
        for line in f:
            if line.startswith("- ") and ":" in line:
                k, v = line[2:].split(":", 1)
                vals[k.strip()] = v.strip()
    return vals


def test_committed_traffic_tracks_the_kernel_source():
    path = os.path.join(ROOT, "profiles", "rs_scatter_small_n16.md")
    vals = _profile_fields(path)
    with open(os.path.join(ROOT, vals["source_file"]), "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()[:16]
    tr = bench.kernel_traffic("rs_scatter", "small_n16")
    if sha == vals["source_sha256"]:
        assert tr == float(vals["dram_bytes_per_launch"])
        # the captured traffic is within 5% of the algorithmic bytes of one pass (24 B per pair
        # over the 9.49e7 pairs of one step's PT2 sort): no re-reads
        assert abs(tr / (24.0 * 16384 * 5792) - 1.0) < 0.05
    else:
        assert tr is None  # stale figures are never reported


def test_peaks_source():
    peaks, kind = bench.load_peaks()
    assert kind in ("measured", "fallback")
    assert peaks["hbm_gbs"] > 1000 and peaks["bf16_tflops"] > 100
    assert bench.whole_job_rate(1e6, 500.0, 4) == 8e6


def test_pt2_screening_default_by_workload(monkeypatch):
    # exact PT2 over C minus S up to 30 orbitals, the paper's screened set above
    for name, eps in (("tiny_n10", 0.0), ("small_n16", 0.0), ("cr2_24e30o", 0.0),
                      ("cr2_48e42o", 1e-6), ("batched", 0.0)):
        monkeypatch.setattr("sys.argv", ["bench.py", "--workload", name])
        assert bench.parse().eps_pt2 == eps
    monkeypatch.setattr("sys.argv", ["bench.py", "--workload", "cr2_48e42o", "--eps-pt2", "0"])
    assert bench.parse().eps_pt2 == 0.0  # an explicit value wins


def test_largest_kernel_issue_figure_tracks_the_kernel_source():
    """The issue-slot fraction of the screened traversal (the bench line's largest kernel) is
    read from its committed ncu summary only while hb.cu is the source it was captured from."""
    path = os.path.join(ROOT, "profiles", "pt2_emit_cr2_48e42o.md")
    vals = _profile_fields(path)
    with open(os.path.join(ROOT, vals["source_file"]), "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()[:16]
    u = bench.kernel_traffic("pt2_emit", "cr2_48e42o", "issue_slots_busy_frac")
    if sha == vals["source_sha256"]:
        assert u == float(vals["issue_slots_busy_frac"]) and 0.0 < u <= 1.0
    else:
        assert u is None


def test_tensor_probe_only_option(monkeypatch):
    """--tensor-probe-only M,N,K (and --probe-mn) select the one-GEMM profiling run."""
    monkeypatch.setattr("sys.argv", ["bench.py", "--tensor-probe-only", "262144,2016,1024"])
    a = bench.parse()
    assert a.tensor_probe_only == "262144,2016,1024" and not a.probe_mn
    assert tuple(int(v) for v in a.tensor_probe_only.split(",")) == (262144, 2016, 1024)
    monkeypatch.setattr("sys.argv", ["bench.py", "--tensor-probe-only", "1024,1024,262144",
                                     "--probe-mn"])
    assert bench.parse().probe_mn
    monkeypatch.setattr("sys.argv", ["bench.py"])
    assert bench.parse().tensor_probe_only is None
