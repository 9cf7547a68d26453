"""Host-side pieces of bench.py: the roofline traffic comes from a committed ncu summary
only while that summary describes the current render source and launch shape."""
import hashlib
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _src_hash():
    src = open(os.path.join(ROOT, "paper_2606_19641_b300", "csrc", "gp_render.cu"), "rb").read()
    return hashlib.sha256(src).hexdigest()


def test_profiled_traffic_follows_the_render_source():
    import re
    for kernel, shape in (("render_kernel", None), ("trace_kernel", "trace")):
        text = open(os.path.join(ROOT, "profiles", kernel + "_uniform_128x128.md")).read()
        m = re.search(r"traffic_bytes_per_launch: (\d+) \(render source sha256 ([0-9a-f]+), "
                      r"shape ([0-9a-z,]+)\)", text)
        assert m, kernel
        b = _bench()
        # the bench reports the captured traffic only for the source the capture was of
        want = int(m.group(1)) if _src_hash().startswith(m.group(2)) else None
        assert b.profiled_traffic(m.group(3), kernel) == want
        assert b.profiled_traffic("1,2,3", kernel) is None  # another launch shape


def test_job_rate_and_reduction_on_one_rank():
    b = _bench()
    # 8192 agents x 100 steps in 200 ms -> 4.096 M agent-steps/s
    assert abs(b.job_rate(8192, 100, 200.0) - 4.096e6) < 1e-3
