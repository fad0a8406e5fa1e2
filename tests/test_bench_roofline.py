"""The bench line's roofline arithmetic and its DRAM-traffic records (host
logic, no GPU): algorithmic bytes per launch of the HBM-bound kernels, the
fraction of the measured peak, and the rule that a captured traffic figure is
reported only while the kernel's sources are the ones it was captured on."""
import hashlib
import json

import pytest

import bench

# the 3D ring workload of the bench step
ROWS, NNZ, NV, NCLS = 44_732_688, 3_967_854_376, 160 * 160 * 104, 84_227


def test_fill_algorithmic_bytes():
    # FP32: 4-byte column + 4-byte chord per nonzero, 8-byte row pointer per row
    bound, work, unit = bench.kernel_model("set_fill_kernel", None, None, None, 3, 3, ROWS, NCLS,
                                           NNZ, NV)
    assert (bound, unit) == ("hbm", "GB/s")
    assert work == 8 * NNZ + 8 * ROWS == 32_100_696_512
    # 16-bit values: 6 bytes per nonzero and a 4-byte FP32 scale per row
    _, work16, _ = bench.kernel_model("set_fill_kernel", None, None, None, 3, 3, ROWS, NCLS, NNZ,
                                      NV, vb=2)
    assert work16 == 6 * NNZ + 4 * ROWS + 8 * ROWS


def test_projector_algorithmic_bytes():
    _, fwd, _ = bench.kernel_model("csr_fwd_wq_kernel", None, None, None, 3, 3, ROWS, NCLS, NNZ,
                                   NV)
    assert fwd == 8 * NNZ + 12 * ROWS + 4 * NV
    for name in ("csr_back_pair_kernel", "csr_back_patch_kernel"):
        _, back, _ = bench.kernel_model(name, None, None, None, 3, 3, ROWS, NCLS, NNZ, NV)
        assert back == 8 * NNZ + 16 * ROWS + 8 * NV


def test_roofline_fraction():
    peaks = {"hbm_gbs": 5000.0}
    r = bench.roofline("csr_fwd_wq_kernel", 10.0, peaks, {"sm_mhz": 2000.0}, None, None, None, 3,
                       3, ROWS, NCLS, NNZ, NV)
    work = 8 * NNZ + 12 * ROWS + 4 * NV
    assert r["bound"] == "hbm" and r["peak_source"] == "measured"
    assert r["achieved"] == pytest.approx(work / 1e9 / 10e-3)
    assert r["frac"] == pytest.approx(r["achieved"] / 5000.0)
    assert r["traffic"] is None  # no capture of this kernel
    # without the measured peaks the fallback copy bandwidth is used, and said
    f = bench.roofline("csr_fwd_wq_kernel", 10.0, {}, {}, None, None, None, 3, 3, ROWS, NCLS,
                       NNZ, NV)
    assert f["peak"] == 6800.0 and f["peak_source"] == "fallback"
    # kernels without a model report only their time
    assert bench.roofline("em_update_kernel", 1.0, peaks, {}, None, None, None, 3, 3, ROWS, NCLS,
                          NNZ, NV) == {"kernel": "em_update_kernel", "ms_per_launch": 1.0,
                                       "bound": None}


def test_traffic_record_follows_its_sources(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    a, b = tmp_path / "a.cu", tmp_path / "b.cuh"
    a.write_bytes(b"kernel body v1")
    b.write_bytes(b"header")
    sha = hashlib.sha1(b"kernel body v1" + b"header").hexdigest()
    rec = {"kx": {"bytes_per_launch": 123, "source": ["a.cu", "b.cuh"], "sha1": sha},
           "ky": {"bytes_per_launch": 7, "source": "a.cu",
                  "sha1": hashlib.sha1(b"kernel body v1").hexdigest()}}
    (tmp_path / "profiles" / "dram_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.kernel_traffic("kx") == 123
    assert bench.kernel_traffic("ky") == 7
    assert bench.kernel_traffic("kz") is None  # never captured
    b.write_bytes(b"header, edited")  # one of the sources changed: the figure is stale
    assert bench.kernel_traffic("kx") is None
    assert bench.kernel_traffic("ky") == 7
    b.unlink()
    assert bench.kernel_traffic("kx") is None


@pytest.mark.parametrize("name", ["set_fill_kernel", "csr_back_patch_kernel"])
def test_committed_records_match_the_sources(name):
    """The DRAM traffic of the bench step's two roofline candidates was captured
    on the committed sources of those kernels."""
    assert bench.kernel_traffic(name) is not None
