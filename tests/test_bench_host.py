"""Host-side logic of bench.py that needs no GPU."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_host_buffer_count():
    b = _bench()
    GB = 1 << 30
    assert b.host_buffer_count(19 * GB, 1, 0) == 2                 # unknown memory: two buffers
    assert b.host_buffer_count(19 * GB, 1, 480 * GB) == 2          # 38 GB of 480
    assert b.host_buffer_count(19 * GB, 8, 480 * GB) == 1          # 304 GB > 288, 152 GB fits
    assert b.host_buffer_count(19 * GB, 16, 480 * GB) == 0         # 304 GB for one buffer each
    assert b.host_buffer_count(11 * GB, 3, 100 * GB) == 1          # 66 GB > 60 % of 100, 33 GB fits
    assert b.host_buffer_count(5 * GB, 6, 100 * GB) == 2           # exactly 60 % fits


def test_clock_summary_median_and_reasons():
    b = _bench()
    c = b.ClockSampler(0)
    c.lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 1980, 2070, 1390.5, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 2040, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage line",
               "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    s = c.summary()
    assert {k: s[k] for k in ("sm_mhz", "sm_max_mhz", "reasons", "samples")} == \
        {"sm_mhz": 2040.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert s["gpu"] == c.id
    c.lines = []
    assert c.summary() is None


def test_gpu_id_follows_visible_devices(monkeypatch):
    # without a CUDA device the sampler names the visible device's own entry (a UUID or
    # a physical index), never this process's ordinal when a mapping is given
    b = _bench()
    monkeypatch.setenv("CUDA_VISIBLE_DEVICES", "GPU-1111-aaaa,GPU-2222-bbbb")
    assert b.gpu_id(1) == "GPU-2222-bbbb"
    monkeypatch.setenv("CUDA_VISIBLE_DEVICES", "5,3")
    assert b.gpu_id(0) == "5"
    monkeypatch.delenv("CUDA_VISIBLE_DEVICES")
    assert b.gpu_id(0) == "0"


def _dram_bytes(profile):
    """(read, write) DRAM bytes of each capture recorded in a committed ncu summary, in
    the order the file lists them."""
    import re
    units = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    text = open(os.path.join(ROOT, "profiles", profile)).read()
    rows = re.findall(r"\| `dram__bytes_(read|write)\.sum` \| (\w+) \| ([\d.]+) \|", text)
    vals = [float(v) * units[u] for _, u, v in rows]
    assert [k for k, _, _ in rows] == ["read", "write"] * (len(rows) // 2)
    return list(zip(vals[0::2], vals[1::2]))


def test_traffic_tables_match_the_profiles():
    # the roofline's `traffic` field comes from bench.py's per-site tables; each entry is
    # a committed capture's DRAM bytes divided by the sites of the captured launch
    b = _bench()
    (rd, wr), = _dram_bytes("k_step_d2q9_wn_fp32_mlp_4096.md")
    assert abs(b.TRAFFIC_PER_SITE[("warp", 4, 0)] * 4096**2 - (rd + wr)) < 1.0
    (rd, wr), = _dram_bytes("k_step_d2q9_tc_fp32_mlp_4096.md")
    assert abs(b.TRAFFIC_PER_SITE[("tcgen05", 2, 0)] * 4096**2 - (rd + wr)) < 1.0
    (r15, w15), (r19, w19) = _dram_bytes("k_step_3d_fp32_256.md")
    assert abs(b.TRAFFIC_PER_SITE_3D[("d3q15_512", 4)] * 256**3 - (r15 + w15)) < 1.0
    assert abs(b.TRAFFIC_PER_SITE_3D[("d3q19_512", 2)] * 256**3 - (r19 + w19)) < 1.0
