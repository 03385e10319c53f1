"""The allocation-free binning entry point (imb_bin_particles_noalloc) against the
context's own binning (imb_get_bins), through the C ABI, on consecutive calls.

It exists for callers that cannot call cudaMalloc (graph capture, hosts that own all
device memory, real-time loops): the test allocates the caller's buffers with PyTorch,
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


def test_noalloc_rejects_more_bins_than_its_scratch():
    from paper_1809_07008_gb300 import binding
    n_side = 32 * 300                      # 300 x 300 bins > IMB_NOALLOC_MAX_BINS
    assert binding.bin_particles_noalloc(0, 0, n_side, n_side, 0, 0, 0) == -1
