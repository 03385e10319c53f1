"""Batched sweep of independent periodic domains (imb_batch_*) against the FP64 oracle run on
each domain by itself.

* Four domains of different sizes (one 75 x 41: rows that end inside a warp's segment), disk
  diameters, solid fractions, relaxation times, body forces and Smagorinsky constants (0 and
  0.1), 300 steps from rest, with one and with two cells per lane: populations of every domain
  (FP32 storage: 1e-6; FP16: 2e-4, the rounding of the stored deviation f - w accumulated over
  the steps) and the per-domain mean drag (FP32: 1e-4 of the drag scale; FP16: 1 %, the storage
  bar the single-lattice tests use).
* A domain without disks (zero drag) beside one with disks, and a batch of a single domain.
* Steps taken two at a time by the replayed graph or one at a time give the same populations
  (bit for bit), the launch-shape search leaves the state as it found it, and steps with the
  shape it chose agree to FP32 rounding.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def imb():
    import paper_1809_07008_gb300 as imb
    imb.load()
    return imb


def _domains():
    return [W.c5_domain(0, 96, 64, 12.0, 0.2, 0.7, 1.0, 11, C_smag=0.0),
            W.c5_domain(1, 128, 96, 16.0, 0.3, 0.52, 30.0, 12),
            W.c5_domain(2, 64, 64, 10.0, 0.12, 1.0, 0.5, 13),
            W.c5_domain(3, 75, 41, 11.0, 0.25, 0.6, 5.0, 14)]


_ORACLE = {}


def _oracle(orc, w, steps):
    key = (w.name, steps)
    if key not in _ORACLE:
        o = orc.Sim(w)
        s = 0.0
        for _ in range(steps):
            o.step(1)
            s += o.forces()[0][:, 0].sum()
        _ORACLE[key] = (o.f(), s / steps)
    return _ORACLE[key]


@pytest.mark.parametrize("storage,tol_f,tol_drag,shape", [("fp32", 1e-6, 1e-4, (256, 1)), ("fp32", 1e-6, 1e-4, (128, 2)),
                                                          ("fp16", 2e-4, 1e-2, (256, 1)), ("fp16", 2e-4, 1e-2, (256, 2))])
def test_batch_matches_oracle_per_domain(orc, imb, storage, tol_f, tol_drag, shape):
    ds = _domains()
    steps = 300
    b = imb.Batch(ds, storage=storage)
    b.set_launch(*shape)
    b.run(steps)
    fx, _ = b.mean_drag()
    for k, w in enumerate(ds):
        fo, drag_o = _oracle(orc, w, steps)
        assert w.n_particles > 0 and abs(drag_o) > 0.0
        assert np.abs(b.populations(k) - fo).max() < tol_f, k
        assert abs(fx[k] - drag_o) < tol_drag * abs(drag_o), (k, fx[k], drag_o)
    b.close()


def test_graph_steps_equal_single_steps_and_autotune_keeps_state(imb):
    ds = _domains()
    b1 = imb.Batch(ds, storage="fp32")
    b1.run(7)                      # three graph replays and one single step
    b2 = imb.Batch(ds, storage="fp32")
    for _ in range(7):
        b2.run(1)
    for k in range(len(ds)):
        assert np.array_equal(b1.populations(k), b2.populations(k))
    before = [b1.populations(k) for k in range(len(ds))]
    blk, cpl, ms = b1.autotune(steps_per_trial=5)
    assert blk in (128, 256, 512) and cpl in (1, 2) and ms > 0.0
    for k in range(len(ds)):
        assert np.array_equal(b1.populations(k), before[k])
    b1.run(3)                      # with the launch shape the search chose
    b2.run(3)
    for k in range(len(ds)):
        assert np.abs(b1.populations(k) - b2.populations(k)).max() < 1e-6
    b1.close()
    b2.close()


def test_set_launch_rejects_bad_shapes_and_keeps_state(imb):
    ds = _domains()
    b = imb.Batch(ds, storage="fp32")
    b.run(5)
    before = [b.populations(k) for k in range(len(ds))]
    for blk, cpl in ((64, 1), (256, 3), (1024, 1)):
        with pytest.raises(imb.ImbError):
            b.set_launch(blk, cpl)
    b.set_launch(128, 2)
    for k in range(len(ds)):
        assert np.array_equal(b.populations(k), before[k])
    b.close()


def test_domain_without_disks_and_single_domain(orc, imb):
    # a domain with no disks (plain forced periodic flow, zero drag) beside one with disks,
    # and a batch of one domain
    plain = W.c5_domain(0, 64, 48, 12.0, 0.2, 0.7, 1.0, 31).with_(x=np.zeros((0, 2)), v=np.zeros((0, 2)),
                                                               omega=np.zeros(0), r=np.zeros(0))
    ds = [plain, W.c5_domain(1, 96, 64, 12.0, 0.2, 0.7, 1.0, 32)]
    for batch in (ds, ds[1:]):
        b = imb.Batch(batch, storage="fp32")
        b.run(100)
        fx, fy = b.mean_drag()
        for k, w in enumerate(batch):
            o = orc.Sim(w)
            o.step(100)
            assert np.abs(b.populations(k) - o.f()).max() < 1e-6
        if batch is ds:
            assert fx[0] == 0.0 and fy[0] == 0.0 and fx[1] != 0.0
        b.close()
