"""Host logic of bench.py that needs no GPU: the clock record taken during the
timed region, from which a run with thermal or hardware slowdown (or clocks
stuck below their maximum) is recognised and rejected."""
import bench


def _summary(text):
    c = bench.Clocks(0)
    c.out = text
    return c.summary()


def test_clock_summary_median_max_and_reasons():
    # clocks.sm, clocks.max.sm, active mask, hw_slowdown, hw_thermal,
    # sw_thermal, sw_power_cap (nvidia-smi csv, noheader, nounits)
    text = "\n".join([
        "2070, 2070, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "2055, 2070, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "1980, 2070, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "2070, 2070, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "2070, 2070, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
    ])
    s = _summary(text)
    assert s["sm_mhz"] == 2070.0
    assert s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    assert s["samples"] == 5
    assert s["gpu"] == bench.gpu_identity(0)


def test_clock_summary_flags_every_slowdown_kind():
    text = "\n".join([
        "1500, 2070, 0x8, Active, Not Active, Not Active, Not Active",
        "1400, 2070, 0x40, Not Active, Active, Not Active, Not Active",
        "1600, 2070, 0x20, Not Active, Not Active, Active, Not Active",
    ])
    s = _summary(text)
    assert s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert s["sm_mhz"] == 1500.0  # median of 1400, 1500, 1600


def test_clock_summary_without_samples_or_with_unreadable_fields():
    assert _summary("") == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
    # a short line is dropped; a field nvidia-smi cannot read is skipped
    s = _summary("2070, 2070\n[N/A], 2070, 0x0, Not Active, Not Active, Not Active, Not Active")
    assert s["samples"] == 1 and s["sm_mhz"] is None and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == []


def test_peaks_measured_file_and_fallback(tmp_path, monkeypatch):
    """The roofline denominators: the measured copy bandwidth and bf16 rate
    when the measured-peaks file is there, else the stated fallback (6.8 TB/s,
    1.9 PFLOP/s), labelled as such."""
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._peaks() == (6800.0, 1900.0, "fallback")
    assert bench._sm_max_mhz() == 2070.0
    (tmp_path / "MEASURED_PEAKS.json").write_text(
        '{"hbm_gbs": 7012.5, "bf16_tflops": 2101.0, "sm_max_mhz": 2062}')
    assert bench._peaks() == (7012.5, 2101.0, "measured")
    assert bench._sm_max_mhz() == 2062.0


def test_gpu_identity_by_uuid(monkeypatch):
    """The clock sampler names its GPU by UUID (CUDA_VISIBLE_DEVICES may
    renumber devices, nvidia-smi's indices never change), falling back to the
    index when torch cannot tell the UUID."""
    import torch

    class P:
        uuid = "0a1b2c3d-0000-1111-2222-333344445555"

    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda i: P())
    assert bench.gpu_identity(0) == "GPU-0a1b2c3d-0000-1111-2222-333344445555"

    def boom(i):
        raise RuntimeError("no device")

    monkeypatch.setattr(torch.cuda, "get_device_properties", boom)
    assert bench.gpu_identity(3) == "3"


def test_algorithmic_bytes_of_the_hbm_bound_steps():
    """The bytes behind the pool and chain HBM fractions, worked out by hand
    for one level: B = 4 (K_p = 16), 1000 pool positions, 400 kept domains,
    300 active ranges, 65536 image pixels."""
    s = {"pool_size_total": 1000, "n_kept": 400, "n_active": 300}
    # image once + 16 B per position + (4 + 2*16 + 32) B per kept domain
    assert bench.pool_bytes(4, s, 65536) == 65536 + 16 * 1000 + 400 * (4 + 32 + 32)
    # per active range: 5n pixels read + 16 K_p operand bytes + 300 B records
    assert bench.chain_bytes(4, s) == 300 * (5 * 16 + 16 * 16 + 300)
    # K_p is the MMA's K step at B = 2 (n = 4 padded to 16)
    assert bench.pool_bytes(2, s, 0) == 16 * 1000 + 400 * (4 + 32 + 32)
