"""bin_and_sort_static: binning and sorting for callers that cannot allocate device memory.

Some callers cannot give the library a workspace: a plugin inside a host application that
owns every device allocation through its own pool, or a real-time frame loop that must
never enter the CUDA allocator.  For them bin_and_sort_static takes its scratch from a
fixed array inside the library.  Its results must be exactly those of bin_and_sort with a
caller workspace (integer outputs: bit-exact).  The check runs two calls in a row, a large
problem and then a smaller one, because every call shares the one scratch array and it
keeps the previous call's contents.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2412_12507_gb300 import abi, render, synth  # noqa: E402

pytestmark = pytest.mark.gpu


def _inputs(seed, n, W, H, tw, th):
    rect, depth = synth.random_rects(seed, n, W, H, max_w=60, max_h=40)
    r = rect.astype(np.int64)
    nt = np.where(r[:, 0] <= r[:, 2], (r[:, 2] // tw - r[:, 0] // tw + 1) * (r[:, 3] // th - r[:, 1] // th + 1), 0)
    dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a, dt)).cuda()  # noqa: E731
    return dev(depth, np.float32), dev(rect, np.int16), dev(nt, np.int32), int(nt.sum())


def _outputs(cap, T):
    return (torch.full((cap,), -1, dtype=torch.int64, device="cuda"),
            torch.full((cap,), -1, dtype=torch.int32, device="cuda"),
            torch.full((T, 2), -1, dtype=torch.int32, device="cuda"),
            torch.zeros(1, dtype=torch.int64, device="cuda"))


def _static_call(n, depth, rect, nt, cam, op, cap, keys, vals, ranges, k_out):
    c, o = abi.make_camera(cam), abi.make_options(op)
    return abi.lib().bin_and_sort_static(n, depth.data_ptr(), rect.data_ptr(), nt.data_ptr(), C.byref(c),
                                         C.byref(o), cap, keys.data_ptr(), vals.data_ptr(), ranges.data_ptr(),
                                         k_out.data_ptr(), torch.cuda.current_stream().cuda_stream)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2412_12507_gb300 import build
    build.build()
    abi.lib()


def test_static_scratch_matches_workspace_version_on_two_calls():
    for seed, n, W, H, tw, th in ((31, 60_000, 1920, 1080, 16, 16), (32, 2_000, 300, 200, 8, 8)):
        cam = synth.camera("pinhole", W, H, fx=float(W))
        op = synth.options(tile_w=tw, tile_h=th)
        depth, rect, nt, K = _inputs(seed, n, W, H, tw, th)
        cap = K + 100
        T = render.tile_count(cam, op)
        # the existing entry point with a caller workspace
        proj = render.Projection(None, None, depth, rect, nt)
        ref = render.bin_and_sort(proj, cam, op, cap, want_keys=True)
        # the no-allocation entry point
        keys, vals, ranges, k_out = _outputs(cap, T)
        st = _static_call(n, depth, rect, nt, cam, op, cap, keys, vals, ranges, k_out)
        assert st == abi.UT_OK, abi.lib().ut_status_string(st)
        torch.cuda.synchronize()
        assert int(k_out.item()) == ref.count() == K
        assert torch.equal(keys[:K], ref.keys[:K])
        assert torch.equal(vals[:K], ref.vals[:K])
        assert torch.equal(ranges, ref.ranges)


def _largest_capacity(n, cam, op):
    """Largest key capacity whose workspace fits the fixed array (host query only)."""
    c, o = abi.make_camera(cam), abi.make_options(op)
    size = lambda cap: abi.lib().ut_bin_workspace_size(n, cap, C.byref(c), C.byref(o))  # noqa: E731
    lo, hi = 0, 1 << 31
    while lo < hi:
        mid = (lo + hi + 1) // 2
        lo, hi = (mid, hi) if size(mid) <= STATIC_BYTES else (lo, mid - 1)
    return lo


STATIC_BYTES = 32 << 20


def test_static_scratch_limit_is_the_documented_one():
    """The header states the largest capacity for 100k particles on a 1080p camera with 16x16
    tiles; at that capacity the call runs and matches bin_and_sort, one key more is refused."""
    W, H, n = 1920, 1080, 100_000
    cam = synth.camera("pinhole", W, H, fx=float(W))
    op = synth.options()
    cap = _largest_capacity(n, cam, op)
    assert cap == 1_446_400
    depth, rect, nt, K = _inputs(34, n, W, H, 16, 16)
    assert K <= cap
    T = render.tile_count(cam, op)
    proj = render.Projection(None, None, depth, rect, nt)
    ref = render.bin_and_sort(proj, cam, op, cap, want_keys=True)
    keys, vals, ranges, k_out = _outputs(cap, T)
    st = _static_call(n, depth, rect, nt, cam, op, cap, keys, vals, ranges, k_out)
    assert st == abi.UT_OK, abi.lib().ut_status_string(st)
    torch.cuda.synchronize()
    assert int(k_out.item()) == ref.count() == K
    assert torch.equal(vals[:K], ref.vals[:K]) and torch.equal(ranges, ref.ranges)
    k_out.fill_(-1)
    ranges.fill_(-1)
    st = _static_call(n, depth, rect, nt, cam, op, cap + 1, keys, vals, ranges, k_out)
    assert st == abi.UT_ERR_CAPACITY
    torch.cuda.synchronize()
    assert int(k_out.item()) == -1 and torch.all(ranges == -1)  # nothing was launched


def test_static_scratch_rejects_sizes_beyond_its_maximum():
    cam = synth.camera("pinhole", 1920, 1080, fx=1920.0)
    op = synth.options()
    depth, rect, nt, K = _inputs(33, 1000, 1920, 1080, 16, 16)
    cap = 10_000_000  # needs far more than the fixed scratch array
    c, o = abi.make_camera(cam), abi.make_options(op)
    assert abi.lib().ut_bin_workspace_size(1000, cap, C.byref(c), C.byref(o)) > STATIC_BYTES
    keys, vals, ranges, k_out = _outputs(16, render.tile_count(cam, op))
    k_out.fill_(-1)  # a sentinel no launch would leave in place
    st = _static_call(1000, depth, rect, nt, cam, op, cap, keys, vals, ranges, k_out)
    assert st == abi.UT_ERR_CAPACITY
    torch.cuda.synchronize()
    assert int(k_out.item()) == -1 and torch.all(ranges == -1)  # nothing was launched
    # a capacity bin_and_sort rejects as invalid is rejected the same way here
    st = _static_call(1000, depth, rect, nt, cam, op, 1 << 32, keys, vals, ranges, k_out)
    assert st == abi.UT_ERR_INVALID_ARG
