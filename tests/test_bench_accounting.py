"""CPU checks of bench.py's roofline arithmetic: the accounting constants, the
choice of the dominant kernel (largest share when the step's kernels run one at
a time), achieved = algorithmic work per launch / launch time, and the ncu DRAM
line being reported only for the CUDA sources it was taken on."""
from types import SimpleNamespace

import pytest

import bench


def test_limb_ntt_accounting():
    # (N/2) log2 N Shoup products x 10 32-bit multiplies
    assert bench.limb_ntt_mults(8192) == 10 * 4096 * 13 == 532480
    assert bench.limb_ntt_mults(4096) == 10 * 2048 * 12
    assert bench.limb_ntt_mults(16384) == 10 * 8192 * 14


def test_headline_mac_work():
    S = SimpleNamespace(ct_in=160, pt=256, ct_out=160, products=2560)
    mults, byts = bench.kernel_work("mac", S, 8192, 3)
    assert mults == 2560 * 2 * 3 * 8192 * 4 == 503316480
    ln = 3 * 8192
    assert byts == 160 * 24 * ln + 256 * 8 * ln + 160 * 24 * ln == 239075328


def test_roofline_picks_the_largest_serial_share_and_divides_by_its_launch_time(monkeypatch):
    S = SimpleNamespace(ct_in=160, pt=256, ct_out=160, products=2560)
    prof = {"mac": (20, 20 * 0.2), "ntt_encode": (20, 20 * 0.1), "mask_poly": (20, 20 * 0.05)}
    serial = {"mac": (3, 3 * 0.15), "ntt_encode": (3, 3 * 0.16), "mask_poly": (3, 3 * 0.5)}
    peaks = {"alu_tmul": 20.0, "alu_source": "derived", "hbm_gbs": 6000.0}
    monkeypatch.setattr(bench, "ncu_traffic", lambda k: None)
    dom, table, roof = bench.roofline(prof, serial, S, 8192, 3, 20, peaks, {})
    # mask_poly has the largest serial share but no multiply accounting: not eligible
    assert dom == "ntt_encode"
    mults = 256 * 3 * bench.limb_ntt_mults(8192)
    assert roof["achieved"] == round(mults / 0.1e-3 / 1e12, 3)
    assert roof["frac"] == round(mults / 0.1e-3 / 1e12 / 20.0, 4)
    assert roof["hbm"]["achieved_gbs"] == round(256 * 8 * 3 * 8192 / 0.1e-3 / 1e9, 1)
    assert table["mac"]["ms_per_launch"] == pytest.approx(0.2)
    assert table["mac"]["ms_per_launch_alone"] == pytest.approx(0.15)
    total = 0.45 + 0.48 + 1.5
    assert table["mask_poly"]["share_alone"] == pytest.approx(1.5 / total)


def test_roofline_rate_from_the_unpipelined_run_when_given(monkeypatch):
    """With two steps in flight a kernel's duration in the main timed run includes
    the time it shares the GPU with the next step's kernels; the dominant kernel's
    rate then comes from the timed run of unpipelined steps."""
    S = SimpleNamespace(ct_in=160, pt=256, ct_out=160, products=2560)
    prof = {"mac": (20, 20 * 0.16), "ntt_encode": (20, 20 * 0.13)}
    serial = {"mac": (3, 3 * 0.145), "ntt_encode": (3, 3 * 0.05)}
    unpiped = {"mac": (20, 20 * 0.144), "ntt_encode": (20, 20 * 0.051)}
    peaks = {"alu_tmul": 20.0, "alu_source": "derived", "hbm_gbs": 6000.0}
    monkeypatch.setattr(bench, "ncu_traffic", lambda k: None)
    dom, table, roof = bench.roofline(prof, serial, S, 8192, 3, 20, peaks, {}, unpiped)
    assert dom == "mac"
    assert roof["duration_from"] == "unpipelined timed run"
    assert roof["achieved"] == round(503316480 / 0.144e-3 / 1e12, 3)
    assert table["mac"]["ms_per_launch"] == pytest.approx(0.16)
    assert table["mac"]["ms_per_launch_unpipelined"] == pytest.approx(0.144)
    dom, table, roof = bench.roofline(prof, serial, S, 8192, 3, 20, peaks, {})
    assert roof["duration_from"] == "timed run"
    assert roof["achieved"] == round(503316480 / 0.16e-3 / 1e12, 3)


def test_ncu_traffic_only_for_the_recorded_sources(tmp_path, monkeypatch):
    digest = bench.csrc_digest()
    prof_dir = tmp_path / "profiles"
    prof_dir.mkdir()
    (prof_dir / "dram_traffic.txt").write_text(
        f"# header\nmac 12345 {digest} workload\nmac 999 0000000000000000 other\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "csrc_digest", lambda: digest)
    assert bench.ncu_traffic("mac") == 12345
    monkeypatch.setattr(bench, "csrc_digest", lambda: "ffffffffffffffff")
    assert bench.ncu_traffic("mac") is None
    assert bench.ncu_traffic("ntt_encode") is None

