"""The benchmark's host-side contract (no GPU): the reference arm's JSON line,
the kernel label each plan variant reports, and the recorded DRAM traffic,
which must belong to the committed sweep sources and the captured variant."""
import json
import os
import subprocess
import sys

import pytest

import __graft_entry__  # noqa: F401  (puts the repo root on the path)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    import bench as b
    return b


@pytest.fixture(scope="module")
def pk():
    from paper_1504_05869_gb300 import build
    build.build()
    import paper_1504_05869_gb300 as pkg
    pkg._pkr.load()
    return pkg


def test_reference_arm_line():
    """`bench.py --impl reference` times the oracle on the host and prints one
    JSON line with the GPU line's metric, unit and direction, its CPU sample
    described, and an e2e object with no host-device copies."""
    oracle_build = subprocess.run([sys.executable, "-c", "import oracle; oracle.build()"],
                                  cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert oracle_build.returncode == 0, oracle_build.stderr[-2000:]
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"].startswith("GLUPS") and line["unit"] == "GLUPS"
    assert line["higher_is_better"] is True and line["value"] > 0
    assert line["steps"] == 1 and line["n_gpus"] == 1
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"]
    assert cb["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "GLUPS",
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert line["config"]["workload"].startswith("poisson3d_256cube_d3q111_n5")


def test_kernel_labels(bench, pk):
    """Staged geometries, the warp-specialised sweep and the two aligned
    x-pairs forms are named in the line's roofline.kernel."""
    nb = pk._pkr.pkr_batch_variant_count(pk.LATTICES["D3Q111"])
    nv = pk._pkr.pkr_variant_count(pk.LATTICES["D3Q111"])
    assert nv == nb + 3
    labels = [bench.kernel_label(pk, v) for v in range(nv)]
    assert all(lab.startswith("sweep_staged_kernel<D3Q111,") for lab in labels[:nb])
    assert labels[nb].startswith("sweep_ws_kernel<D3Q111,")
    assert "refill after the pair" in labels[nb + 1]
    assert labels[nb + 2].startswith("sweep_pair_kernel<D3Q111,") and "early refill" in labels[-1]


@pytest.mark.parametrize("precision", ["fx64", "fp64"])
def test_recorded_traffic_matches_the_sources(bench, precision, monkeypatch):
    """The committed 128^3 traffic capture, scaled to 256^3, is reported only
    for the variant it was taken on and only while the sweep sources hash to
    the value recorded with it; it lies within 2 % of the algorithmic bytes."""
    monkeypatch.setattr(bench, "PRECISION", precision)
    t = bench.recorded_traffic(8)
    assert t is not None, "sweep sources changed since the traffic capture"
    algorithmic = 256 ** 3 * (2 * 111 * 8 + 8)
    assert abs(t / algorithmic - 1) < 0.02
    assert bench.recorded_traffic(2) is None
    monkeypatch.setattr(bench, "PRECISION", "fp32")
    assert bench.recorded_traffic(8) is None
