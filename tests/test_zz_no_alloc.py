"""pic_bin_particles_noalloc: the box binning for callers that cannot let a
library allocate device memory (work issued inside an open stream capture,
frameworks that own all device memory through their own pool, loops that must
never reach the allocator).  Its only scratch is a fixed array compiled into
libpic, so its results must match the allocating pic_bin_particles exactly --
including on a second call, which finds the first call's cursors still in that
array.  Collected last on purpose, so that a stop at the first failure has
already run every other test."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _inputs(seed, dim, n, box, dx, npart):
    import torch
    rng = np.random.default_rng(seed)
    L = [n[a] * dx[a] for a in range(3)]
    x = rng.uniform(0, L[0], npart)
    y = rng.uniform(0, L[1], npart) if dim == 3 else None
    z = rng.uniform(0, L[2], npart)
    t = lambda a: None if a is None else torch.as_tensor(a, device="cuda")  # noqa: E731
    return t(x), t(y), t(z)


def _run(fn, dim, n, box, dx, x, y, z):
    import torch
    from paper_2104_11385_gb300 import sim as S
    nb = int(np.prod([n[a] // box[a] for a in range(3)]))
    off = torch.full((nb + 1,), -7, dtype=torch.int64, device="cuda")
    perm = torch.full((x.numel(),), -7, dtype=torch.int64, device="cuda")
    S.bin_particles(dim, n, box, dx, x, y, z, off, perm, fn=fn)
    torch.cuda.synchronize()
    return off.cpu().numpy(), perm.cpu().numpy()


def _same(a, b):
    off_a, perm_a = a
    off_b, perm_b = b
    assert np.array_equal(off_a, off_b)
    for k in range(len(off_a) - 1):  # same members per box; the order inside a box is free
        sl = slice(off_a[k], off_a[k + 1])
        assert np.array_equal(np.sort(perm_a[sl]), np.sort(perm_b[sl]))


def test_noalloc_matches_allocating_entry_point_on_two_calls_in_a_row():
    cases = [
        # first call: many boxes, dense; second: fewer boxes, so stale cursors
        # of the first call sit in the shared scratch
        (3, (64, 64, 64), (8, 8, 8), (0.25, 0.25, 0.25), 300_000, 1),
        (2, (96, 1, 64), (16, 1, 16), (0.3, 1.0, 0.2), 50_001, 2),
    ]
    for dim, n, box, dx, npart, seed in cases:
        x, y, z = _inputs(seed, dim, n, box, dx, npart)
        ref = _run("pic_bin_particles", dim, n, box, dx, x, y, z)
        got = _run("pic_bin_particles_noalloc", dim, n, box, dx, x, y, z)
        _same(got, ref)
        assert ref[0][-1] == npart


def test_noalloc_rejects_more_boxes_than_its_scratch():
    import torch
    from paper_2104_11385_gb300 import _lib as L
    from paper_2104_11385_gb300 import sim as S
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    off = torch.zeros(8, dtype=torch.int64, device="cuda")
    perm = torch.zeros(4, dtype=torch.int64, device="cuda")
    n = (2048, 1024, 2)  # 2^22 boxes of 1 cell
    with pytest.raises(L.PicError) as ei:
        S.bin_particles(3, n, (1, 1, 1), (1.0, 1.0, 1.0), x, x, x, off, perm, fn="pic_bin_particles_noalloc")
    assert ei.value.status == L.PIC_EINVAL
    assert "scratch" in str(ei.value)


def test_noalloc_call_captured_in_a_cuda_graph():
    """The call allocates and synchronises nothing, so once its first call on
    the device has run (the scratch address lookup), it can be captured into a
    CUDA graph in the global capture mode; the graph's replays give the
    allocating call's result, also after the inputs are rewritten in place."""
    import torch
    from paper_2104_11385_gb300 import sim as S
    dim, n, box, dx, npart = 3, (32, 32, 32), (8, 8, 8), (0.25, 0.25, 0.25), 100_000
    nb = int(np.prod([n[a] // box[a] for a in range(3)]))
    x, y, z = _inputs(7, dim, n, box, dx, npart)
    off = torch.full((nb + 1,), -7, dtype=torch.int64, device="cuda")
    perm = torch.full((npart,), -7, dtype=torch.int64, device="cuda")
    S.bin_particles(dim, n, box, dx, x, y, z, off, perm, fn="pic_bin_particles_noalloc")  # outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        S.bin_particles(dim, n, box, dx, x, y, z, off, perm, stream=torch.cuda.current_stream().cuda_stream,
                        fn="pic_bin_particles_noalloc")
    for seed in (7, 8):
        if seed != 7:
            x2, y2, z2 = _inputs(seed, dim, n, box, dx, npart)
            x.copy_(x2)
            y.copy_(y2)
            z.copy_(z2)
        ref = _run("pic_bin_particles", dim, n, box, dx, x, y, z)
        off.fill_(-7)
        perm.fill_(-7)
        g.replay()
        torch.cuda.synchronize()
        _same((off.cpu().numpy(), perm.cpu().numpy()), ref)
