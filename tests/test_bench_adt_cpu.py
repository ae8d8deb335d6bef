"""The transfer model of the bench's ADT section (Sec. III-B, Eq. 1), pinned to
what the paper states about it, and the traffic-record lookup of the roofline."""
import json

import pytest


def _b():
    import bench
    return bench


def test_eq1_three_packets_saves_two_transfer_pairs():
    # Sec. III-B: three packets take 3(T_PS + T_DKE + T_PR) with SDT and
    # T_PS + 3 T_DKE + T_PR with ADT, a saving of 2(T_PS + T_PR)
    b = _b()
    for t_ps, t_dke, t_pr in ((1.0, 5.0, 2.0), (3.0, 1.0, 4.0), (0.5, 0.5, 0.5)):
        sdt = 3 * (t_ps + t_dke + t_pr)
        adt = t_ps + 3 * t_dke + t_pr
        assert sdt - adt == pytest.approx(2 * (t_ps + t_pr))
        assert b.eq1_speedup(3, t_ps, t_dke, t_pr) == pytest.approx(sdt / adt)


def test_eq1_regimes():
    b = _b()
    # when T_PS + T_PR = T_DKE the speedup is 2N / (N + 1), about 2
    for n in (1, 2, 8, 1000):
        assert b.eq1_speedup(n, 1.0, 3.0, 2.0) == pytest.approx(2 * n / (n + 1))
    # one packet: nothing to overlap
    assert b.eq1_speedup(1, 1.0, 7.0, 2.0) == pytest.approx(1.0)
    # vanishing kernel time: the speedup tends to N
    assert b.eq1_speedup(16, 1.0, 1e-9, 1.0) == pytest.approx(16.0, rel=1e-6)


def test_pipeline_form_equals_eq1_when_the_kernel_is_slowest():
    b = _b()
    for n in (1, 3, 8):
        assert b.pipeline_speedup(n, 1.0, 5.0, 2.0) == pytest.approx(b.eq1_speedup(n, 1.0, 5.0, 2.0))
    # with copies slower than the kernel the pipeline form is the smaller one,
    # bounded by the sum of the stages over the slowest one
    n, t_ps, t_dke, t_pr = 8, 84.0, 16.0, 96.0
    p = b.pipeline_speedup(n, t_ps, t_dke, t_pr)
    assert p < b.eq1_speedup(n, t_ps, t_dke, t_pr)
    assert 1.0 < p < (t_ps + t_dke + t_pr) / max(t_ps, t_dke, t_pr)


def test_traffic_record_lookup(tmp_path, monkeypatch):
    b = _b()
    (tmp_path / "profiles").mkdir()
    h = b.kernel_sources_hash()
    recs = {"records": [
        {"kernel": "k_decode_stream<63, 1, 128, 3, 32, 1>", "dram_bytes_read": 10, "dram_bytes_write": 5,
         "sources_sha256": h},
        {"kernel": "k_decode_stream<63, 1, 128, 2, 32, 1>", "dram_bytes_read": 10, "dram_bytes_write": 7,
         "sources_sha256": "stale"},
    ]}
    (tmp_path / "profiles" / "roofline_traffic_n63.json").write_text(json.dumps(recs))
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    monkeypatch.setattr(b, "kernel_sources_hash", lambda: h)
    assert b.recorded_traffic("k_decode_stream<63, 1, 128, 3, 32, 1>") == 15
    assert b.recorded_traffic("k_decode_stream<63, 1, 128, 2, 32, 1>") is None  # sources changed since
    assert b.recorded_traffic("k_decode_stream<63, 1, 192, 2, 32, 1>") is None  # no record

