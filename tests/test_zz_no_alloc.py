"""The allocation-free binning entry point (imb_bin_particles_noalloc) against the
context's own binning (imb_get_bins), through the C ABI, on consecutive calls.

It exists for callers that cannot call cudaMalloc (hosts that own all device memory,
real-time loops): the test allocates the caller's buffers with PyTorch,
the entry point itself allocates nothing and keeps its scratch in a fixed device array
shared by all calls.  Bins are integer bookkeeping, so the outputs must be identical.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _noalloc_bins(binding, torch, w, stream):
    nb = ((w.nx + 31) // 32) * ((w.ny + 31) // 32)
    x = torch.from_numpy(np.ascontiguousarray(w.x.reshape(-1))).cuda()
    start = torch.full((nb + 1,), -7, dtype=torch.int32, device="cuda")
    ids = torch.full((max(w.n_particles, 1),), -7, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    rc = binding.bin_particles_noalloc(x.data_ptr(), w.n_particles, w.nx, w.ny, start.data_ptr(),
                                       ids.data_ptr(), stream.cuda_stream)
    assert rc == 0
    stream.synchronize()
    return start.cpu().numpy(), ids.cpu().numpy()[:w.n_particles]


def test_noalloc_bins_match_context_bins_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    import paper_1809_07008_gb300 as imb
    from paper_1809_07008_gb300 import binding
    imb.load()
    stream = torch.cuda.Stream()
    # two different layouts in a row, then the first again: the shared scratch is cleared
    # by every call, so each result must equal the context's bins for that layout
    layouts = [W.c3sub(steps=0, nx=512, ny=512), W.c2(steps=0), W.c3sub(steps=0, nx=512, ny=512)]
    for w in layouts:
        lat = imb.Lattice.from_workload(w)
        ref_start, ref_ids = lat.bins()
        start, ids = _noalloc_bins(binding, torch, w, stream)
        assert np.array_equal(start, ref_start)
        assert np.array_equal(ids, ref_ids)
        lat.close()


def test_noalloc_allocates_nothing():
    # neither PyTorch's allocator nor the device's free memory moves across calls (the first
    # call may load the library's module, which brings the fixed scratch array with it)
    torch = pytest.importorskip("torch")
    import paper_1809_07008_gb300 as imb
    from paper_1809_07008_gb300 import binding
    imb.load()
    stream = torch.cuda.Stream()
    w = W.c3sub(steps=0, nx=512, ny=512)
    _noalloc_bins(binding, torch, w, stream)
    x = torch.from_numpy(np.ascontiguousarray(w.x.reshape(-1))).cuda()
    start = torch.zeros(((512 // 32) ** 2 + 1,), dtype=torch.int32, device="cuda")
    ids = torch.zeros((w.n_particles,), dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    before = (torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0])
    for _ in range(3):
        assert binding.bin_particles_noalloc(x.data_ptr(), w.n_particles, w.nx, w.ny, start.data_ptr(),
                                             ids.data_ptr(), stream.cuda_stream) == 0
    stream.synchronize()
    assert (torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]) == before


def test_noalloc_bin_limit():
    # real buffers, so that only the bin count can refuse the call: 300 x 300 bins exceed
    # IMB_NOALLOC_MAX_BINS (65 536) and are refused; 256 x 256 bins (8192 x 8192 cells, the
    # largest the scratch holds) run and equal the context's bins
    torch = pytest.importorskip("torch")
    import paper_1809_07008_gb300 as imb
    from paper_1809_07008_gb300 import binding
    imb.load()
    stream = torch.cuda.Stream()
    x = torch.full((2,), 5.0, dtype=torch.float64, device="cuda")
    start = torch.zeros((300 * 300 + 1,), dtype=torch.int32, device="cuda")
    ids = torch.zeros((1,), dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    n_side = 32 * 300
    assert binding.bin_particles_noalloc(x.data_ptr(), 1, n_side, n_side, start.data_ptr(), ids.data_ptr(),
                                         stream.cuda_stream) == -1
    w = W.c3(steps=0, n=3000, nx=8192, ny=8192)
    lat = imb.Lattice.from_workload(w)
    ref_start, ref_ids = lat.bins()
    lat.close()
    bins_start, bins_ids = _noalloc_bins(binding, torch, w, stream)
    assert len(bins_start) == 256 * 256 + 1
    assert np.array_equal(bins_start, ref_start) and np.array_equal(bins_ids, ref_ids)
