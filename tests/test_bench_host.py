"""Host-side byte accounting of bench.py (no GPU): the algorithmic bytes per
node of the whole step and of each kernel class, against the figures derived
from what each kernel must read and write once."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_step_bytes():
    b = _bench()
    # populations in and out once + n,u out, n in, g2 out, n,u,g2 in
    assert b.bytes_alg(0) == 2 * 19 * 4 + 16 + 4 + 4 + 20 == 196
    assert b.bytes_alg(1) == 2 * 19 * 2 + 44 == 120


def test_kernel_bytes_add_up():
    b = _bench()
    for storage, s in ((0, 4), (1, 2)):
        fused = b.kernel_bytes(storage, True)
        two = b.kernel_bytes(storage, False)
        # the fused step: ball (n in, g2 out), force (n,u,g2 in, F out), collide-stream-moments
        step_fused = fused["ball_g2"] + fused["force"] + fused["collide_stream"]
        assert step_fused == 2 * 19 * s + 8 + 36 + 32 + 16
        # above the algorithmic minimum by F through memory (+32) and the fields read again (+16)
        assert step_fused - b.bytes_alg(storage) == 48
        # the two-pass step re-reads the populations in its moments pass
        step_two = two["moments"] + two["ball_g2"] + two["force"] + two["collide_stream"]
        assert step_two - step_fused == 19 * s + 24 - 16


def test_measured_traffic_covers_the_dominant_kernels():
    b = _bench()
    t = b.TRAFFIC_B_PER_NODE_F32
    for k in ("collide_stream_fused", "collide_stream", "force", "ball_g2", "moments"):
        assert t[k] > 0
    # DRAM traffic of the fused pass stays within 10 % of its algorithmic bytes
    assert abs(t["collide_stream_fused"] / b.kernel_bytes(0, True)["collide_stream"] - 1) < 0.1
