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
