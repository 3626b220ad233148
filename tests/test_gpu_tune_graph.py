"""The streaming-product autotuner and the graph-replayed product: the tuned
launch configuration changes results only by the order of FP32 sums (and a
grid change not at all); graph replays give the plain path's bits and read
the arrays' current contents."""
import numpy as np
import pytest

import cavities as cv
from gpu_common import rad

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def handle():
    r = rad()
    verts = cv.icosphere(3)
    h = r.rad_build_htree(verts, leaf_size=32, eta_adm=1.0)
    r.rad_compress_aca(h, 1e-5, 64, "partial", "f32", "f32")
    yield r, h, verts.shape[0]
    h.free()


@pytest.mark.parametrize("factor", ["f32", "bf16"])
def test_autotune_changes_no_result(handle, factor):
    r, h, n = handle
    r.rad_compress_aca(h, 1e-5, 64, "partial", factor, "f32")
    rng = np.random.default_rng(11)
    x1 = rng.uniform(0.5, 1.5, n)
    x2 = rng.uniform(0.5, 1.5, (n, 2))
    y1, y2 = r.rad_hmatvec(h, x1), r.rad_hmatvec(h, x2)
    assert r.rad_htree_get_stats(h)["tuned"] == 0
    cfg = r.rad_htree_autotune(h)
    st = r.rad_htree_get_stats(h)
    assert st["tuned"] == 1 and cfg["stream_rows"] in (64, 128, 256) and cfg["product_path"] in (0, 1)
    for k in ("grid_a1", "grid_b1", "grid_a2", "grid_b2"):
        assert cfg[k] >= 0
    # the grid policy changes nothing; the item rows change only the order of
    # the FP32 sums
    assert np.abs(r.rad_hmatvec(h, x1) - y1).max() <= 2e-6 * np.abs(y1).max()
    assert np.abs(r.rad_hmatvec(h, x2) - y2).max() <= 2e-6 * np.abs(y2).max()
    ya = r.rad_hmatvec(h, x1)
    np.testing.assert_array_equal(r.rad_hmatvec(h, x1), ya)
    # recompression resets the choice
    r.rad_compress_aca(h, 1e-5, 64, "partial", factor, "f32")
    assert r.rad_htree_get_stats(h)["tuned"] == 0


def test_graph_replay_reads_current_arrays(handle):
    r, h, n = handle
    r.rad_compress_aca(h, 1e-5, 64, "partial", "f32", "f32")
    dev = torch.device("cuda", 0)
    x = torch.as_tensor(np.random.default_rng(2).uniform(0.5, 1.5, n), dtype=torch.float32, device=dev)
    y = torch.empty(n, dtype=torch.float32, device=dev)
    r.rad_hmatvec(h, x, y)
    ref = y.clone()
    c0 = r.rad_launch_count()
    for _ in range(3):           # capture on the 2nd call, replays after
        y.zero_()
        r.rad_hmatvec(h, x, y)
        torch.cuda.synchronize()
        assert torch.equal(y, ref)
    per_call = (r.rad_launch_count() - c0) / 3
    assert per_call >= 2
    x.mul_(2.0)                  # exact scaling: the replay must see it
    r.rad_hmatvec(h, x, y)
    torch.cuda.synchronize()
    assert torch.equal(y, 2.0 * ref)
    y2 = torch.empty_like(y)     # other output array: ordinary path
    r.rad_hmatvec(h, x, y2)
    torch.cuda.synchronize()
    assert torch.equal(y2, y)


def test_graph_inside_a_caller_capture(handle):
    """A caller capturing its own stream gets plain launches recorded."""
    r, h, n = handle
    r.rad_compress_aca(h, 1e-5, 64, "partial", "f32", "f32")
    dev = torch.device("cuda", 0)
    x = torch.ones(n, dtype=torch.float32, device=dev)
    y = torch.empty(n, dtype=torch.float32, device=dev)
    r.rad_hmatvec(h, x, y)
    ref = y.clone()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    y.zero_()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
        r.rad_hmatvec(h, x, y, stream=s.cuda_stream)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(y, ref)
