"""Host-side arithmetic of bench.py's JSON line (no GPU): the HBM view of a
kernel, the peak lookup and its fallback, and the kernel-source hash that
decides whether a committed ncu traffic figure still applies."""
import json

import pytest

import bench


def test_hbm_view_arithmetic():
    v = bench.hbm_view(2.0e9, 1.0)          # 2 GB in 1 ms = 2000 GB/s
    assert v["unit"] == "GB/s"
    assert v["achieved"] == pytest.approx(2000.0)
    assert v["frac"] == pytest.approx(2000.0 / bench.HBM_PEAK_GBS)
    assert bench.hbm_view(1.0e9, 0.0) is None
    assert bench.hbm_view(1.0e9, None) is None


def test_measured_peak_fallback(tmp_path, monkeypatch):
    # a missing key falls back and says so
    assert bench._measured_peak("no_such_peak", 123.0) == (123.0, "fallback")
    # a file with the key is read as measured
    f = tmp_path / "MEASURED_PEAKS.json"
    f.write_text(json.dumps({"hbm_gbs": 4321.0}))
    monkeypatch.setattr(bench.os.path, "dirname", lambda _p: str(tmp_path))
    assert bench._measured_peak("hbm_gbs", 1.0) == (4321.0, "measured")
    assert bench._measured_peak("bf16_tflops", 7.0) == (7.0, "fallback")


def test_kernel_source_hash_tracks_the_kernel_text():
    span = bench.MPK_KERNEL_TEXT
    text = f"prefix\n{span[0]}\nbody A\n{span[1]}\nsuffix"
    h = bench.kernel_source_hash(text=text, span=span)
    assert h == bench.kernel_source_hash(text=text.replace("prefix", "other prefix"), span=span)
    assert h != bench.kernel_source_hash(text=text.replace("body A", "body B"), span=span)
    # the committed kernel still contains the span bench.py hashes
    assert len(bench.kernel_source_hash()) == 16


def test_timed_solves_run_without_phase_events():
    """The timed solves run with the library's per-phase timing off (its
    events break the chain of dependent launches); everything else in the
    options is the phase pass's."""
    P = pytest.importorskip("paper_1701_03989_gb300")
    o = P.make_options(method="adaptive", basis="chebyshev", s_max=16, eps_target=1e-12, lam=(0.01, 1.0),
                       timing=True, gram_fp64=True)
    u = bench.untimed(P, o)
    assert o.flags & P.ASCG_FLAG_TIMING
    assert not u.flags & P.ASCG_FLAG_TIMING
    assert u.flags == o.flags & ~P.ASCG_FLAG_TIMING
    assert (u.method, u.basis, u.s_max, u.eps_target) == (o.method, o.basis, o.s_max, o.eps_target)
    assert o.flags & P.ASCG_FLAG_TIMING  # the original is left as it was
